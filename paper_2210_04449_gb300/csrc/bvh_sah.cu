// Binned surface-area-heuristic topology for the Sec. 2.2 ray casts (the
// paper leaves the ray-tracing structure open).
//
// Top-down: the triangles of a node (a contiguous range of leaf positions)
// are split where the surface-area heuristic (MacDonald & Booth 1990) is
// lowest, cost = half-area(left box) x left count + half-area(right box) x
// right count, evaluated over 32 bins of the range's centroid bounds per
// axis (binning as in Wald 2007).  Every range is split down to single
// triangles.  Node ids need no allocation: the node whose right child starts
// at leaf position s is node s - 1 (each boundary between neighbouring leaves
// belongs to exactly one node), so the tree has the layout of the Morton
// tree: [nt - 1] nodes, [nt] leaves, any node may be the root.
//
// Three tiers by range size m:
//  * m > SAH_CH: level-synchronous over chunks of SAH_CH positions.
//    k_sah_bin bins a chunk in shared memory and merges into the range's
//    bins with global atomics (and keeps the chunk's histogram);
//    k_sah_split (a warp per range) picks the split and every chunk's output
//    offset; k_sah_partition scatters stably into the other order buffer.
//  * 32 < m <= SAH_CH: one block per range (k_sah_block), boxes in shared
//    memory, the same binned split down to ranges of 32;
//  * 2 <= m <= 32: one warp per range, the exact heuristic over every split
//    of the centroids sorted along each axis (bitonic sort in registers).
// Float min/max merges go through an order-preserving map to uint32, so
// every merge is exact and independent of order: the build is
// deterministic, whatever order the atomics land in.
#include <math_constants.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace rtsdf {

namespace {

constexpr int NB = 32;                        // bins per axis (one per lane)
constexpr int BW = 7;                         // words per bin: count, lo xyz, hi xyz
constexpr int SAH_BIN_WORDS = 3 * NB * BW;
constexpr int SAH_CH = 1024;                  // chunk size, largest block range
constexpr int SAH_THREADS = 256;
constexpr int SAH_ITEMS = SAH_CH / SAH_THREADS;
constexpr int SAH_WARPS = SAH_THREADS / 32;
constexpr int WARP_MAX = 32;                  // largest range of the exact warp build
constexpr int BLK_STACK = 48;                 // disjoint ranges > 32 in 1024: at most 31
constexpr int WLIST_CAP = SAH_CH / 2;         // disjoint ranges >= 2 in 1024
constexpr int WSTACK = 32;                    // disjoint ranges >= 2 in 32: at most 16
constexpr unsigned FULL = 0xFFFFFFFFu;

static_assert(SAH_ITEMS * SAH_THREADS == SAH_CH, "one chunk per block pass");

// big range (m > SAH_CH) of one level
struct SahTask {
    int32_t b, e, parent, side;
    int32_t buf, chunk0, nchunk, axis;   // buf: order buffer holding the range
    int32_t split, nl, child[2];         // split: first right bin (-1: median)
    uint32_t cb[6];                      // centroid bounds, ordered uint: lo xyz, hi xyz
    int32_t pad[2];
};
static_assert(sizeof(SahTask) == 80, "task record");

// range for the block tier: [b, e), parent node, side | buf << 1
struct SahRange {
    int32_t b, e, parent, sb;
};

__device__ __forceinline__ uint32_t f2o(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}
__device__ __forceinline__ float cen(float lo, float hi) { return __fmul_rn(0.5f, __fadd_rn(lo, hi)); }
__device__ __forceinline__ float half_area3(const float lo[3], const float hi[3]) {
    const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return dx * dy + dy * dz + dz * dx;
}
__device__ __forceinline__ uint32_t bin_init(int i) {
    const int w = i % BW;
    return w == 0 ? 0u : (w < 4 ? 0xFFFFFFFFu : 0u);
}

struct BinMap {
    float lo[3], scale[3];
};
__device__ __forceinline__ BinMap bin_map(const float clo[3], const float chi[3]) {
    BinMap m;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        m.lo[a] = clo[a];
        const float ext = chi[a] - clo[a];
        float s = ext > 0.f ? (float)NB / ext : 0.f;
        if (!(s <= 3.0e38f)) s = 0.f;       // a denormal extent: treat as flat
        m.scale[a] = s;
    }
    return m;
}
__device__ __forceinline__ int bin_of(const BinMap& m, int a, float c) {
    const int k = (int)((c - m.lo[a]) * m.scale[a]);
    return min(max(k, 0), NB - 1);
}

struct Choice {
    float cost;
    int axis, split, nl;   // axis -1: no axis separates the range
};

// Lane l reads bin l of each axis; the split after bin l puts bins 0..l left.
// Ties go to the smaller bin, then the smaller axis.  All 32 lanes call.
__device__ Choice warp_choose(const uint32_t* bins, int lane) {
    Choice best{CUDART_INF_F, -1, -1, 0};
    for (int a = 0; a < 3; a++) {
        const uint32_t* p = bins + (a * NB + lane) * BW;
        const uint32_t cnt = p[0];
        float plo[3], phi[3], slo[3], shi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            plo[k] = slo[k] = cnt ? o2f(p[1 + k]) : CUDART_INF_F;
            phi[k] = shi[k] = cnt ? o2f(p[4 + k]) : -CUDART_INF_F;
        }
        uint32_t pc = cnt, sc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t up = __shfl_up_sync(FULL, pc, o), dn = __shfl_down_sync(FULL, sc, o);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float ul = __shfl_up_sync(FULL, plo[k], o), uh = __shfl_up_sync(FULL, phi[k], o);
                const float dl = __shfl_down_sync(FULL, slo[k], o), dh = __shfl_down_sync(FULL, shi[k], o);
                if (lane >= o) {
                    plo[k] = fminf(plo[k], ul);
                    phi[k] = fmaxf(phi[k], uh);
                }
                if (lane + o < 32) {
                    slo[k] = fminf(slo[k], dl);
                    shi[k] = fmaxf(shi[k], dh);
                }
            }
            if (lane >= o) pc += up;
            if (lane + o < 32) sc += dn;
        }
        // right side of the split after bin `lane`: the suffix from lane + 1
        const uint32_t rc = __shfl_down_sync(FULL, sc, 1);
        float rlo[3], rhi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            rlo[k] = __shfl_down_sync(FULL, slo[k], 1);
            rhi[k] = __shfl_down_sync(FULL, shi[k], 1);
        }
        float cost = CUDART_INF_F;
        if (lane < NB - 1 && pc > 0 && rc > 0)
            cost = half_area3(plo, phi) * (float)pc + half_area3(rlo, rhi) * (float)rc;
        float bc = cost;
        int bl = lane;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float c2 = __shfl_xor_sync(FULL, bc, o);
            const int l2 = __shfl_xor_sync(FULL, bl, o);
            if (c2 < bc || (c2 == bc && l2 < bl)) {
                bc = c2;
                bl = l2;
            }
        }
        const uint32_t nl = __shfl_sync(FULL, pc, bl);
        if (bc < best.cost) {
            best.cost = bc;
            best.axis = a;
            best.split = bl + 1;
            best.nl = (int)nl;
        }
    }
    return best;
}

// Where a build writes its topology.  A parent id >= 0 is a node, -1 the
// tree's root, <= -2 the root of segment -2 - parent (per-segment builds).
// A top-level build over segments (child_of set) names its nodes through
// node_ids (local id -> node) and makes each of its leaves the subtree
// child_of[item] of the listed segment `item`.
struct Links {
    BNode* nodes;
    int32_t* leaf_parent;
    int32_t* root;
    int32_t* seg_root;
    const int32_t* node_ids;
    const int32_t* child_of;
};

__device__ __forceinline__ void hook(const Links& L, int parent, int side, int child) {
    if (parent >= 0) {
        if (side) L.nodes[parent].d.y = child;
        else L.nodes[parent].d.x = child;
    } else if (parent == -1) {
        *L.root = child;
    } else {
        L.seg_root[-2 - parent] = child;
    }
}

__device__ __forceinline__ void make_node(const Links& L, int id, int parent, int side) {
    L.nodes[id].d.z = parent;
    L.nodes[id].d.w = 0;
    hook(L, parent, side, id);
}

// Leaf at global position pos, or in a top-level build the subtree of item.
__device__ __forceinline__ void make_leaf(const Links& L, int parent, int side, int pos, int item) {
    if (L.child_of) {
        const int c = L.child_of[item];
        hook(L, parent, side, c);
        if (c >= 0) L.nodes[c].d.z = parent;
        else L.leaf_parent[~c] = parent;
    } else {
        hook(L, parent, side, ~pos);
        L.leaf_parent[pos] = parent;
    }
}

// Exclusive block-wide sum (all SAH_THREADS threads call).
__device__ __forceinline__ int block_excl(int v, int* s_warp, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < SAH_WARPS; w++) {
        const int s = s_warp[w];
        if (w < warp) off += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return off + inc - v;
}

// ------------------------------------------------------------- setup

__global__ void k_sah_root(SahTask* t, int4* chunks, uint32_t* bins, SahRange* blist, int32_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nch = (n + SAH_CH - 1) / SAH_CH;
    if (i == 0) {
        SahTask r;
        r.b = 0; r.e = n; r.parent = -1; r.side = 0;
        r.buf = 0; r.chunk0 = 0; r.nchunk = nch; r.axis = -1;
        r.split = -1; r.nl = 0; r.child[0] = r.child[1] = -1;
        for (int k = 0; k < 3; k++) {
            r.cb[k] = 0xFFFFFFFFu;
            r.cb[3 + k] = 0u;
        }
        r.pad[0] = r.pad[1] = 0;
        t[0] = r;
        if (n <= SAH_CH) blist[0] = SahRange{0, n, -1, 0};
    }
    if (n > SAH_CH) {
        if (i < nch) chunks[i] = make_int4(0, i * SAH_CH, min(SAH_CH, n - i * SAH_CH), 0);
        if (i < SAH_BIN_WORDS) bins[i] = bin_init(i);
    }
}

// Per triangle: its box (unpadded); for a single-root build also the
// identity order and the root's centroid bounds (ord, root: nullptr for a
// segment build).
__global__ void __launch_bounds__(SAH_THREADS) k_sah_prims(const float* __restrict__ verts,
                                                           const int32_t* __restrict__ tris, int32_t n,
                                                           float4* __restrict__ pbox, int32_t* __restrict__ ord,
                                                           SahTask* root) {
    __shared__ float s_red[SAH_WARPS][6];
    const int i = blockIdx.x * SAH_THREADS + threadIdx.x;
    float r[6] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
    if (i < n) {
        const float* p0 = verts + 3 * (int64_t)tris[3 * (int64_t)i];
        const float* p1 = verts + 3 * (int64_t)tris[3 * (int64_t)i + 1];
        const float* p2 = verts + 3 * (int64_t)tris[3 * (int64_t)i + 2];
        float lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lo[a] = fminf(p0[a], fminf(p1[a], p2[a]));
            hi[a] = fmaxf(p0[a], fmaxf(p1[a], p2[a]));
            const float c = cen(lo[a], hi[a]);
            r[a] = c;
            r[3 + a] = c;
        }
        pbox[2 * (int64_t)i] = make_float4(lo[0], lo[1], lo[2], 0.f);
        pbox[2 * (int64_t)i + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
        if (ord) ord[i] = i;
    }
    if (!root) return;                          // block-uniform: segment builds set their own bounds
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            r[k] = fminf(r[k], __shfl_xor_sync(FULL, r[k], o));
            r[3 + k] = fmaxf(r[3 + k], __shfl_xor_sync(FULL, r[3 + k], o));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 6; k++) s_red[warp][k] = r[k];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        float v = s_red[0][k];
        for (int w = 1; w < SAH_WARPS; w++) v = k < 3 ? fminf(v, s_red[w][k]) : fmaxf(v, s_red[w][k]);
        if (v == v && fabsf(v) <= 3.4e38f) {   // skip the empty value of an all-idle block
            if (k < 3) atomicMin(&root->cb[k], f2o(v));
            else atomicMax(&root->cb[k], f2o(v));
        }
    }
}

// Centroid bounds of the first level's big ranges of a segment build (one
// block per range) and their bins reset.
__global__ void __launch_bounds__(SAH_THREADS) k_sah_task_init(SahTask* tasks, const int32_t* __restrict__ ord,
                                                               const float4* __restrict__ pbox, uint32_t* bins) {
    __shared__ float s_red[SAH_WARPS][6];
    SahTask& T = tasks[blockIdx.x];
    float r[6] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
    for (int p = T.b + threadIdx.x; p < T.e; p += SAH_THREADS) {
        const int32_t t = ord[p];
        const float4 lo = pbox[2 * (int64_t)t], hi = pbox[2 * (int64_t)t + 1];
        const float c[3] = {cen(lo.x, hi.x), cen(lo.y, hi.y), cen(lo.z, hi.z)};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            r[k] = fminf(r[k], c[k]);
            r[3 + k] = fmaxf(r[3 + k], c[k]);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            r[k] = fminf(r[k], __shfl_xor_sync(FULL, r[k], o));
            r[3 + k] = fmaxf(r[3 + k], __shfl_xor_sync(FULL, r[3 + k], o));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 6; k++) s_red[warp][k] = r[k];
    for (int i = threadIdx.x; i < SAH_BIN_WORDS; i += SAH_THREADS)
        bins[(size_t)blockIdx.x * SAH_BIN_WORDS + i] = bin_init(i);
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        float v = s_red[0][k];
        for (int w = 1; w < SAH_WARPS; w++) v = k < 3 ? fminf(v, s_red[w][k]) : fmaxf(v, s_red[w][k]);
        T.cb[k] = f2o(v);                       // a big range is never empty
    }
}

// A top-level tree over a single segment: the segment's subtree is the root.
__global__ void k_sah_top_single(const int32_t* child_of, BNode* nodes, int32_t* leaf_parent, int32_t* root) {
    const int c = child_of[0];
    *root = c;
    if (c >= 0) nodes[c].d.z = -1;
    else leaf_parent[~c] = -1;
}

// ------------------------------------------------------------- big ranges

__global__ void __launch_bounds__(SAH_THREADS) k_sah_bin(const int4* __restrict__ chunks,
                                                         const SahTask* __restrict__ tasks,
                                                         const int32_t* __restrict__ ord0,
                                                         const int32_t* __restrict__ ord1,
                                                         const float4* __restrict__ pbox, uint32_t* bins,
                                                         uint32_t* __restrict__ hist) {
    __shared__ uint32_t sb[SAH_BIN_WORDS];
    const int4 ch = chunks[blockIdx.x];        // (task, start, length)
    const SahTask& T = tasks[ch.x];
    for (int i = threadIdx.x; i < SAH_BIN_WORDS; i += SAH_THREADS) sb[i] = bin_init(i);
    float clo[3], chi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        clo[a] = o2f(T.cb[a]);
        chi[a] = o2f(T.cb[3 + a]);
    }
    const BinMap m = bin_map(clo, chi);
    const int32_t* ord = T.buf ? ord1 : ord0;
    __syncthreads();
    for (int i = threadIdx.x; i < ch.z; i += SAH_THREADS) {
        const int32_t t = ord[ch.y + i];
        const float4 lo = pbox[2 * (int64_t)t], hi = pbox[2 * (int64_t)t + 1];
        const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            uint32_t* p = sb + (a * NB + bin_of(m, a, cen(l[a], h[a]))) * BW;
            atomicAdd(p, 1u);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                atomicMin(p + 1 + k, f2o(l[k]));
                atomicMax(p + 4 + k, f2o(h[k]));
            }
        }
    }
    __syncthreads();
    uint32_t* gb = bins + (size_t)ch.x * SAH_BIN_WORDS;
    for (int i = threadIdx.x; i < SAH_BIN_WORDS; i += SAH_THREADS) {
        const int w = i % BW;
        const uint32_t cnt = sb[i - w];
        if (w == 0) hist[(size_t)blockIdx.x * 3 * NB + i / BW] = cnt;
        if (cnt == 0) continue;
        if (w == 0) atomicAdd(gb + i, cnt);
        else if (w < 4) atomicMin(gb + i, sb[i]);
        else atomicMax(gb + i, sb[i]);
    }
}

// One warp per big range: split choice, node links, chunk output offsets,
// and the children (leaf, block range or next-level big range).
// counters: [0] next tasks, [1] next chunks, [2] block ranges, [3] overflow.
__global__ void __launch_bounds__(SAH_THREADS) k_sah_split(SahTask* tasks, int32_t ntask, const uint32_t* bins,
                                                           const uint32_t* __restrict__ hist,
                                                           const int4* __restrict__ chunks,
                                                           int32_t* __restrict__ left_off, Links L, SahTask* next,
                                                           int4* next_chunks, uint32_t* next_bins, SahRange* blist,
                                                           int32_t* counters, int32_t cap_task, int32_t cap_chunk,
                                                           int32_t cap_blist) {
    const int w = (int)((blockIdx.x * (unsigned)SAH_THREADS + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= ntask) return;                    // warp-uniform
    SahTask& T = tasks[w];
    const int b = T.b, e = T.e, m = e - b;
    const Choice ch = warp_choose(bins + (size_t)w * SAH_BIN_WORDS, lane);
    const int nl = ch.axis < 0 ? m / 2 : ch.nl;
    // left items before each chunk (chunks of a range are in position order)
    int carry = 0;
    for (int k0 = 0; k0 < T.nchunk; k0 += 32) {
        const int k = k0 + lane;
        int lc = 0;
        if (k < T.nchunk) {
            const int4 cr = chunks[T.chunk0 + k];
            if (ch.axis < 0) {
                lc = min(max(nl - (cr.y - b), 0), cr.z);
            } else {
                const uint32_t* h = hist + (size_t)(T.chunk0 + k) * 3 * NB + ch.axis * NB;
                for (int j = 0; j < ch.split; j++) lc += (int)h[j];
            }
        }
        int inc = lc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += u;
        }
        if (k < T.nchunk) left_off[T.chunk0 + k] = carry + inc - lc;
        carry += __shfl_sync(FULL, inc, 31);
    }
    const int id = b + nl - 1;
    int child[2] = {-1, -1};
    for (int s = 0; s < 2; s++) {
        const int cb = s ? b + nl : b, ce = s ? e : b + nl, cm = ce - cb;
        if (cm == 1) {
            if (lane == 0) make_leaf(L, id, s, cb, -1);
        } else if (cm <= SAH_CH) {
            if (lane == 0) {
                const int q = atomicAdd(counters + 2, 1);
                if (q < cap_blist) blist[q] = SahRange{cb, ce, id, s | ((T.buf ^ 1) << 1)};
                else atomicOr(counters + 3, 1);
            }
        } else {
            const int nch = (cm + SAH_CH - 1) / SAH_CH;
            int q = 0, c0 = 0;
            if (lane == 0) {
                q = atomicAdd(counters, 1);
                c0 = atomicAdd(counters + 1, nch);
            }
            q = __shfl_sync(FULL, q, 0);
            c0 = __shfl_sync(FULL, c0, 0);
            if (q < cap_task && c0 + nch <= cap_chunk) {
                child[s] = q;
                if (lane == 0) {
                    SahTask r;
                    r.b = cb; r.e = ce; r.parent = id; r.side = s;
                    r.buf = T.buf ^ 1; r.chunk0 = c0; r.nchunk = nch; r.axis = -1;
                    r.split = -1; r.nl = 0; r.child[0] = r.child[1] = -1;
                    for (int k = 0; k < 3; k++) {
                        r.cb[k] = 0xFFFFFFFFu;
                        r.cb[3 + k] = 0u;
                    }
                    r.pad[0] = r.pad[1] = 0;
                    next[q] = r;
                }
                for (int k = lane; k < nch; k += 32)
                    next_chunks[c0 + k] = make_int4(q, cb + k * SAH_CH, min(SAH_CH, ce - (cb + k * SAH_CH)), 0);
                for (int i = lane; i < SAH_BIN_WORDS; i += 32) next_bins[(size_t)q * SAH_BIN_WORDS + i] = bin_init(i);
            } else if (lane == 0) {
                atomicOr(counters + 3, 1);
            }
        }
    }
    if (lane == 0) {
        make_node(L, id, T.parent, T.side);
        T.axis = ch.axis;
        T.split = ch.split;
        T.nl = nl;
        T.child[0] = child[0];
        T.child[1] = child[1];
    }
}

// Stable scatter of a chunk to the other order buffer; leaves get their
// final position; big children get their centroid bounds.
__global__ void __launch_bounds__(SAH_THREADS) k_sah_partition(const int4* __restrict__ chunks,
                                                               const SahTask* __restrict__ tasks,
                                                               const int32_t* __restrict__ left_off, int32_t* ord0,
                                                               int32_t* ord1, const float4* __restrict__ pbox,
                                                               int32_t* __restrict__ order_final, SahTask* next) {
    __shared__ int s_warp[SAH_WARPS];
    __shared__ uint32_t s_cb[2][6];
    const int4 ch = chunks[blockIdx.x];
    const SahTask& T = tasks[ch.x];
    const int32_t* src = T.buf ? ord1 : ord0;
    int32_t* dst = T.buf ? ord0 : ord1;
    if (threadIdx.x < 12) s_cb[threadIdx.x / 6][threadIdx.x % 6] = (threadIdx.x % 6) < 3 ? 0xFFFFFFFFu : 0u;
    float clo[3], chi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        clo[a] = o2f(T.cb[a]);
        chi[a] = o2f(T.cb[3 + a]);
    }
    const BinMap m = bin_map(clo, chi);
    const int axis = T.axis, split = T.split, nl = T.nl, b = T.b, msz = T.e - T.b;
    const int i0 = threadIdx.x * SAH_ITEMS;
    int32_t t[SAH_ITEMS];
    float c[SAH_ITEMS][3];
    bool left[SAH_ITEMS];
    int nleft = 0;
#pragma unroll
    for (int j = 0; j < SAH_ITEMS; j++) {
        const int i = i0 + j;
        left[j] = false;
        t[j] = -1;
        if (i < ch.z) {
            t[j] = src[ch.y + i];
            const float4 lo = pbox[2 * (int64_t)t[j]], hi = pbox[2 * (int64_t)t[j] + 1];
            c[j][0] = cen(lo.x, hi.x);
            c[j][1] = cen(lo.y, hi.y);
            c[j][2] = cen(lo.z, hi.z);
            left[j] = axis < 0 ? (ch.y + i - b) < nl : bin_of(m, axis, c[j][axis]) < split;
            nleft += left[j];
        }
    }
    int total = 0;
    const int lrank0 = block_excl(nleft, s_warp, total);   // also orders the s_cb init
    const int lo_base = b + left_off[blockIdx.x];
    const int ro_base = b + nl + (ch.y - b - left_off[blockIdx.x]);
    int lr = lrank0, rr = min(i0, ch.z) - lrank0;
    const bool need_cb = T.child[0] >= 0 || T.child[1] >= 0;
#pragma unroll
    for (int j = 0; j < SAH_ITEMS; j++) {
        if (t[j] < 0) continue;
        const int pos = left[j] ? lo_base + lr++ : ro_base + rr++;
        dst[pos] = t[j];
        if ((left[j] ? nl : msz - nl) == 1) order_final[pos] = t[j];
        if (need_cb && T.child[left[j] ? 0 : 1] >= 0) {
            uint32_t* p = s_cb[left[j] ? 0 : 1];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                atomicMin(p + k, f2o(c[j][k]));
                atomicMax(p + 3 + k, f2o(c[j][k]));
            }
        }
    }
    if (!need_cb) return;                      // block-uniform
    __syncthreads();
    if (threadIdx.x < 12) {
        const int s = threadIdx.x / 6, k = threadIdx.x % 6;
        const int q = T.child[s];
        const uint32_t v = s_cb[s][k];
        if (q >= 0 && v != (k < 3 ? 0xFFFFFFFFu : 0u)) {
            if (k < 3) atomicMin(&next[q].cb[k], v);
            else atomicMax(&next[q].cb[k], v);
        }
    }
}

// ------------------------------------------------------------- block ranges

struct BlockSmem {
    float lo[3][SAH_CH], hi[3][SAH_CH];   // by slot (load order)
    int32_t tri[SAH_CH];                  // triangle of each slot
    uint16_t perm[SAH_CH], tmp[SAH_CH];   // slot at each position
    uint32_t bins[SAH_BIN_WORDS];
    SahRange stack[BLK_STACK];
    SahRange wlist[WLIST_CAP];
    SahRange wstack[SAH_WARPS][WSTACK];
    float red[SAH_WARPS][6];
    int scan[SAH_WARPS];
    Choice choice;
    int top, nw, bad;
};

// Exact heuristic for a range of <= 32 positions, one warp; sub-ranges on a
// warp-private stack.  Positions are local to the block's range (global
// position = gb + local).
__device__ void warp_exact(BlockSmem& S, SahRange r0, int gb, const Links& L, int lane, SahRange* st) {
    int top = 1;
    if (lane == 0) st[0] = r0;
    __syncwarp();
    for (int guard = 0; top > 0 && guard < 2 * WARP_MAX; guard++) {
        const SahRange r = st[top - 1];
        top--;
        __syncwarp();
        const int lb = r.b, mm = r.e - r.b;
        int nl = 1;
        if (mm > 2) {
            const int slot = lane < mm ? (int)S.perm[lb + lane] : 0;
            float c[3], lo[3], hi[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                lo[k] = lane < mm ? S.lo[k][slot] : CUDART_INF_F;
                hi[k] = lane < mm ? S.hi[k][slot] : -CUDART_INF_F;
                c[k] = lane < mm ? cen(lo[k], hi[k]) : CUDART_INF_F;
            }
            float bestc = CUDART_INF_F;
            int bestj = 0, bestidx = lane;
            for (int a = 0; a < 3; a++) {
                float key = c[a];
                int idx = lane;
#pragma unroll
                for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const float ok = __shfl_xor_sync(FULL, key, j);
                        const int oi = __shfl_xor_sync(FULL, idx, j);
                        const bool other_less = ok < key || (ok == key && oi < idx);
                        const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                        if (keep_min ? other_less : !other_less) {
                            key = ok;
                            idx = oi;
                        }
                    }
                float plo[3], phi[3], slo[3], shi[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    plo[k] = slo[k] = __shfl_sync(FULL, lo[k], idx);
                    phi[k] = shi[k] = __shfl_sync(FULL, hi[k], idx);
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1)
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const float ul = __shfl_up_sync(FULL, plo[k], o), uh = __shfl_up_sync(FULL, phi[k], o);
                        const float dl = __shfl_down_sync(FULL, slo[k], o), dh = __shfl_down_sync(FULL, shi[k], o);
                        if (lane >= o) {
                            plo[k] = fminf(plo[k], ul);
                            phi[k] = fmaxf(phi[k], uh);
                        }
                        if (lane + o < 32) {
                            slo[k] = fminf(slo[k], dl);
                            shi[k] = fmaxf(shi[k], dh);
                        }
                    }
                float rlo[3], rhi[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    rlo[k] = __shfl_down_sync(FULL, slo[k], 1);
                    rhi[k] = __shfl_down_sync(FULL, shi[k], 1);
                }
                float cost = CUDART_INF_F;
                if (lane < mm - 1)
                    cost = half_area3(plo, phi) * (float)(lane + 1) + half_area3(rlo, rhi) * (float)(mm - 1 - lane);
                // equal costs: the split nearest the middle, then the smaller one
                float bc = cost;
                int bl = lane;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const float c2 = __shfl_xor_sync(FULL, bc, o);
                    const int l2 = __shfl_xor_sync(FULL, bl, o);
                    const int d1 = abs(2 * bl + 2 - mm), d2 = abs(2 * l2 + 2 - mm);
                    if (c2 < bc || (c2 == bc && (d2 < d1 || (d2 == d1 && l2 < bl)))) {
                        bc = c2;
                        bl = l2;
                    }
                }
                if (bc < bestc) {
                    bestc = bc;
                    bestj = bl;
                    bestidx = idx;
                }
            }
            nl = bestj + 1;
            // position lb + lane takes the slot that sorted to rank `lane`
            const int ns = __shfl_sync(FULL, slot, bestidx);
            if (lane < mm) S.perm[lb + lane] = (uint16_t)ns;
            __syncwarp();
        }
        const int id = L.node_ids ? L.node_ids[lb + nl - 1] : gb + lb + nl - 1;
        if (lane == 0) make_node(L, id, r.parent, r.sb & 1);
        for (int s = 0; s < 2; s++) {
            const int cb = s ? lb + nl : lb, ce = s ? r.e : lb + nl;
            if (ce - cb == 1) {
                if (lane == 0) make_leaf(L, id, s, gb + cb, S.tri[S.perm[cb]]);
            } else {
                if (lane == 0 && top < WSTACK) st[top] = SahRange{cb, ce, id, s};
                top++;
            }
        }
        if (top > WSTACK) {                   // cannot happen: disjoint ranges of >= 2 in 32
            if (lane == 0) S.bad = 1;
            top = WSTACK;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(SAH_THREADS) k_sah_block(const SahRange* __restrict__ blist,
                                                           const int32_t* __restrict__ ord0,
                                                           const int32_t* __restrict__ ord1,
                                                           const float4* __restrict__ pbox,
                                                           int32_t* __restrict__ order_final, Links L,
                                                           int32_t* counters) {
    extern __shared__ __align__(16) unsigned char sah_smem[];
    BlockSmem& S = *reinterpret_cast<BlockSmem*>(sah_smem);
    const SahRange R = blist[blockIdx.x];
    const int gb = R.b, m = R.e - R.b;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t* ord = (R.sb >> 1) ? ord1 : ord0;
    for (int i = tid; i < m; i += SAH_THREADS) {
        const int32_t t = ord[gb + i];
        const float4 l = pbox[2 * (int64_t)t], h = pbox[2 * (int64_t)t + 1];
        S.lo[0][i] = l.x; S.lo[1][i] = l.y; S.lo[2][i] = l.z;
        S.hi[0][i] = h.x; S.hi[1][i] = h.y; S.hi[2][i] = h.z;
        S.tri[i] = t;
        S.perm[i] = (uint16_t)i;
    }
    if (tid == 0) {
        S.top = 0;
        S.nw = 0;
        S.bad = 0;
        const SahRange r{0, m, R.parent, R.sb & 1};
        if (m > WARP_MAX) S.stack[S.top++] = r;
        else S.wlist[S.nw++] = r;
    }
    __syncthreads();
    for (int guard = 0; guard < 2 * SAH_CH; guard++) {
        if (S.top == 0) break;                 // block-uniform: read after a barrier
        const SahRange r = S.stack[S.top - 1];
        const int lb = r.b, le = r.e, mm = le - lb;
        // centroid bounds of the range; bins reset
        float cb[6] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
        for (int p = lb + tid; p < le; p += SAH_THREADS) {
            const int s = S.perm[p];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float c = cen(S.lo[k][s], S.hi[k][s]);
                cb[k] = fminf(cb[k], c);
                cb[3 + k] = fmaxf(cb[3 + k], c);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                cb[k] = fminf(cb[k], __shfl_xor_sync(FULL, cb[k], o));
                cb[3 + k] = fmaxf(cb[3 + k], __shfl_xor_sync(FULL, cb[3 + k], o));
            }
        if (lane == 0)
            for (int k = 0; k < 6; k++) S.red[warp][k] = cb[k];
        for (int i = tid; i < SAH_BIN_WORDS; i += SAH_THREADS) S.bins[i] = bin_init(i);
        __syncthreads();
        if (tid == 0) S.top--;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float v = S.red[0][k];
            for (int w = 1; w < SAH_WARPS; w++) v = k < 3 ? fminf(v, S.red[w][k]) : fmaxf(v, S.red[w][k]);
            cb[k] = v;
        }
        const BinMap bm = bin_map(cb, cb + 3);
        for (int p = lb + tid; p < le; p += SAH_THREADS) {
            const int s = S.perm[p];
            float l[3], h[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                l[k] = S.lo[k][s];
                h[k] = S.hi[k][s];
            }
#pragma unroll
            for (int a = 0; a < 3; a++) {
                uint32_t* q = S.bins + (a * NB + bin_of(bm, a, cen(l[a], h[a]))) * BW;
                atomicAdd(q, 1u);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    atomicMin(q + 1 + k, f2o(l[k]));
                    atomicMax(q + 4 + k, f2o(h[k]));
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            Choice c = warp_choose(S.bins, lane);
            if (c.axis < 0) c.nl = mm / 2;
            if (lane == 0) S.choice = c;
        }
        __syncthreads();
        const Choice c = S.choice;
        const int nl = c.nl;
        // stable partition of positions [lb, le)
        const int i0 = tid * SAH_ITEMS;
        bool left[SAH_ITEMS];
        int nleft = 0;
#pragma unroll
        for (int j = 0; j < SAH_ITEMS; j++) {
            const int i = i0 + j;
            left[j] = false;
            if (i < mm) {
                const int s = S.perm[lb + i];
                left[j] = c.axis < 0 ? i < nl : bin_of(bm, c.axis, cen(S.lo[c.axis][s], S.hi[c.axis][s])) < c.split;
                nleft += left[j];
            }
        }
        int total = 0;
        const int lr0 = block_excl(nleft, S.scan, total);
        int lr = lr0, rr = min(i0, mm) - lr0;
#pragma unroll
        for (int j = 0; j < SAH_ITEMS; j++) {
            const int i = i0 + j;
            if (i < mm) S.tmp[lb + (left[j] ? lr++ : nl + rr++)] = S.perm[lb + i];
        }
        __syncthreads();
        for (int p = lb + tid; p < le; p += SAH_THREADS) S.perm[p] = S.tmp[p];
        if (tid == 0) {
            const int id = L.node_ids ? L.node_ids[lb + nl - 1] : gb + lb + nl - 1;
            make_node(L, id, r.parent, r.sb & 1);
            for (int s = 0; s < 2; s++) {
                const int cb0 = s ? lb + nl : lb, ce = s ? le : lb + nl, cm = ce - cb0;
                const SahRange ch{cb0, ce, id, s};
                if (cm == 1) {
                    make_leaf(L, id, s, gb + cb0, S.tri[S.tmp[cb0]]);   // tmp: this range's new order
                } else if (cm <= WARP_MAX) {
                    if (S.nw < WLIST_CAP) S.wlist[S.nw++] = ch;
                    else S.bad = 1;
                } else {
                    if (S.top < BLK_STACK) S.stack[S.top++] = ch;
                    else S.bad = 1;
                }
            }
        }
        __syncthreads();
    }
    for (int q = warp; q < S.nw; q += SAH_WARPS) warp_exact(S, S.wlist[q], gb, L, lane, S.wstack[warp]);
    __syncthreads();
    if (order_final)
        for (int i = tid; i < m; i += SAH_THREADS) order_final[gb + i] = S.tri[S.perm[i]];
    if (tid == 0 && (S.bad || S.top != 0)) atomicOr(counters + 3, 2);
}

}  // namespace

size_t sah_scratch_bytes(int64_t n) {
    const int64_t cap_task = n / (SAH_CH + 1) + 2;
    const int64_t cap_chunk = 2 * (n / SAH_CH) + 4;
    const int64_t cap_blist = n / 2 + 2;
    return sizeof(float4) * 2 * n + sizeof(int32_t) * 3 * n + sizeof(uint32_t) * 3 * NB * cap_chunk +
           sizeof(int32_t) * cap_chunk + sizeof(SahTask) * 2 * cap_task + sizeof(int4) * 2 * cap_chunk +
           sizeof(uint32_t) * SAH_BIN_WORDS * 2 * cap_task + sizeof(SahRange) * cap_blist + 16 * sizeof(int32_t) +
           16 * 256;   // alignment slack
}

namespace {

struct SahArena {
    float4* pbox;
    int32_t *ord0, *ord1, *loff, *counters;
    uint32_t* hist;
    SahTask* tasks[2];
    int4* chunks[2];
    uint32_t* bins[2];
    SahRange* blist;
    int32_t cap_task, cap_chunk, cap_blist;
};

cudaError_t carve(void* scratch, int32_t n, SahArena& A) {
    A.cap_task = n / (SAH_CH + 1) + 2;
    A.cap_chunk = 2 * (n / SAH_CH) + 4;
    A.cap_blist = n / 2 + 2;
    unsigned char* p = (unsigned char*)scratch;
    auto take = [&](size_t bytes) {
        void* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    A.pbox = (float4*)take(sizeof(float4) * 2 * (size_t)n);
    A.ord0 = (int32_t*)take(sizeof(int32_t) * (size_t)n);
    A.ord1 = (int32_t*)take(sizeof(int32_t) * (size_t)n);
    A.hist = (uint32_t*)take(sizeof(uint32_t) * 3 * NB * (size_t)A.cap_chunk);
    A.loff = (int32_t*)take(sizeof(int32_t) * (size_t)A.cap_chunk);
    for (int k = 0; k < 2; k++) A.tasks[k] = (SahTask*)take(sizeof(SahTask) * (size_t)A.cap_task);
    for (int k = 0; k < 2; k++) A.chunks[k] = (int4*)take(sizeof(int4) * (size_t)A.cap_chunk);
    for (int k = 0; k < 2; k++) A.bins[k] = (uint32_t*)take(sizeof(uint32_t) * SAH_BIN_WORDS * (size_t)A.cap_task);
    A.blist = (SahRange*)take(sizeof(SahRange) * (size_t)A.cap_blist);
    A.counters = (int32_t*)take(16 * sizeof(int32_t));
    return (size_t)(p - (unsigned char*)scratch) > sah_scratch_bytes(n) ? cudaErrorInvalidValue : cudaSuccess;
}

cudaError_t block_attr(rtsdf_ctx* c) {
    static bool attr_set[64] = {};             // per device ordinal
    const int dv = c->device >= 0 && c->device < 64 ? c->device : 0;
    if (!attr_set[dv]) {
        cudaError_t e = cudaFuncSetAttribute(k_sah_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(BlockSmem));
        if (e != cudaSuccess) return e;
        attr_set[dv] = true;
    }
    return cudaSuccess;
}

// The level loop over big ranges, then the block ranges; ntask / nchunk /
// nblock describe the first level (already in A).
cudaError_t run_levels(rtsdf_ctx* c, SahArena& A, const Links& L, int32_t* order, int32_t ntask, int32_t nchunk,
                       int32_t nblock) {
    cudaError_t e;
    int cur = 0;
    for (int level = 0; ntask > 0; level++) {
        if (level >= 4096) return cudaErrorUnknown;   // sizes shrink every level; only a fault gets here
        if ((e = cudaMemsetAsync(A.counters, 0, 2 * sizeof(int32_t), c->stream))) return e;
        RTSDF_LAUNCH(c, k_sah_bin, (unsigned)nchunk, SAH_THREADS, 0, A.chunks[cur], A.tasks[cur], A.ord0, A.ord1,
                     A.pbox, A.bins[cur], A.hist);
        RTSDF_LAUNCH(c, k_sah_split, (unsigned)((ntask + SAH_WARPS - 1) / SAH_WARPS), SAH_THREADS, 0, A.tasks[cur],
                     ntask, A.bins[cur], A.hist, A.chunks[cur], A.loff, L, A.tasks[cur ^ 1], A.chunks[cur ^ 1],
                     A.bins[cur ^ 1], A.blist, A.counters, A.cap_task, A.cap_chunk, A.cap_blist);
        RTSDF_LAUNCH(c, k_sah_partition, (unsigned)nchunk, SAH_THREADS, 0, A.chunks[cur], A.tasks[cur], A.loff, A.ord0,
                     A.ord1, A.pbox, order, A.tasks[cur ^ 1]);
        int32_t h[4] = {0, 0, 0, 0};
        if ((e = cudaGetLastError())) return e;
        if ((e = cudaMemcpyAsync(h, A.counters, sizeof(h), cudaMemcpyDeviceToHost, c->stream))) return e;
        if ((e = cudaStreamSynchronize(c->stream))) return e;
        if (h[3] != 0 || h[0] > A.cap_task || h[1] > A.cap_chunk || h[2] > A.cap_blist) return cudaErrorUnknown;
        ntask = h[0];
        nchunk = h[1];
        nblock = h[2];
        cur ^= 1;
    }
    if (nblock > 0)
        RTSDF_LAUNCH(c, k_sah_block, (unsigned)nblock, SAH_THREADS, sizeof(BlockSmem), A.blist, A.ord0, A.ord1,
                     A.pbox, order, L, A.counters);
    if ((e = cudaGetLastError())) return e;
    int32_t bad = 0;
    if ((e = cudaMemcpyAsync(&bad, A.counters + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream))) return e;
    if ((e = cudaStreamSynchronize(c->stream))) return e;
    return bad ? cudaErrorUnknown : cudaSuccess;   // a capacity guard fired: cannot happen for a valid range
}

}  // namespace

cudaError_t sah_topology(rtsdf_ctx* c, void* scratch, int32_t* order) {
    Bvh& bv = c->bvh;
    const int32_t n = (int32_t)bv.nt;
    SahArena A;
    cudaError_t e = carve(scratch, n, A);
    if (!e) e = block_attr(c);
    if (!e) e = cudaMemsetAsync(A.counters, 0, 16 * sizeof(int32_t), c->stream);
    if (e) return e;
    const int nch0 = (n + SAH_CH - 1) / SAH_CH;
    const int init_threads = nch0 > SAH_BIN_WORDS ? nch0 : SAH_BIN_WORDS;
    RTSDF_LAUNCH(c, k_sah_root, (unsigned)((init_threads + 255) / 256), 256, 0, A.tasks[0], A.chunks[0], A.bins[0],
                 A.blist, n);
    RTSDF_LAUNCH(c, k_sah_prims, (unsigned)((n + SAH_THREADS - 1) / SAH_THREADS), SAH_THREADS, 0, c->verts, c->tris,
                 n, A.pbox, A.ord0, A.tasks[0]);
    const Links L{bv.nodes, bv.leaf_parent, bv.root, nullptr, nullptr, nullptr};
    return run_levels(c, A, L, order, n > SAH_CH ? 1 : 0, nch0, n > SAH_CH ? 0 : 1);
}

cudaError_t sah_segments(rtsdf_ctx* c, void* scratch, int32_t* order, const int32_t* order_in,
                         const int32_t* bounds, int32_t nseg, int32_t* seg_root) {
    Bvh& bv = c->bvh;
    const int32_t n = (int32_t)bv.nt;
    SahArena A;
    cudaError_t e = carve(scratch, n, A);
    if (!e) e = block_attr(c);
    if (e) return e;
    // the first level, laid out on the host
    std::vector<SahTask> tasks;
    std::vector<int4> chunks;
    std::vector<SahRange> blist;
    std::vector<int32_t> root0((size_t)nseg, 0);
    for (int32_t k = 0; k < nseg; k++) {
        const int32_t b = bounds[k], en = bounds[k + 1], m = en - b;
        if (m == 1) {
            root0[(size_t)k] = ~b;                // a one-triangle segment is its own leaf
        } else if (m <= SAH_CH) {
            blist.push_back(SahRange{b, en, -2 - k, 0});
        } else {
            SahTask t;
            memset(&t, 0, sizeof(t));
            t.b = b; t.e = en; t.parent = -2 - k; t.side = 0; t.buf = 0;
            t.chunk0 = (int32_t)chunks.size();
            t.nchunk = (m + SAH_CH - 1) / SAH_CH;
            t.axis = -1; t.split = -1; t.child[0] = t.child[1] = -1;
            for (int q = 0; q < t.nchunk; q++)
                chunks.push_back(make_int4((int)tasks.size(), b + q * SAH_CH, std::min(SAH_CH, en - (b + q * SAH_CH)), 0));
            tasks.push_back(t);
        }
    }
    if ((int64_t)tasks.size() > A.cap_task || (int64_t)chunks.size() > A.cap_chunk ||
        (int64_t)blist.size() > A.cap_blist)
        return cudaErrorInvalidValue;   // cannot happen: the segments partition [0, n)
    int32_t h0[16] = {0};
    h0[2] = (int32_t)blist.size();
    if ((e = cudaMemcpyAsync(A.counters, h0, sizeof(h0), cudaMemcpyHostToDevice, c->stream))) return e;
    if ((e = cudaMemcpyAsync(seg_root, root0.data(), sizeof(int32_t) * (size_t)nseg, cudaMemcpyHostToDevice,
                             c->stream)))
        return e;
    if (!tasks.empty() &&
        ((e = cudaMemcpyAsync(A.tasks[0], tasks.data(), sizeof(SahTask) * tasks.size(), cudaMemcpyHostToDevice,
                              c->stream)) ||
         (e = cudaMemcpyAsync(A.chunks[0], chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice,
                              c->stream))))
        return e;
    if (!blist.empty() && (e = cudaMemcpyAsync(A.blist, blist.data(), sizeof(SahRange) * blist.size(),
                                               cudaMemcpyHostToDevice, c->stream)))
        return e;
    if ((e = cudaMemcpyAsync(A.ord0, order_in, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    RTSDF_LAUNCH(c, k_sah_prims, (unsigned)((n + SAH_THREADS - 1) / SAH_THREADS), SAH_THREADS, 0, c->verts, c->tris,
                 n, A.pbox, (int32_t*)nullptr, (SahTask*)nullptr);
    if (!tasks.empty())
        RTSDF_LAUNCH(c, k_sah_task_init, (unsigned)tasks.size(), SAH_THREADS, 0, A.tasks[0], A.ord0, A.pbox, A.bins[0]);
    // one-triangle segments are final at once
    if ((e = cudaMemcpyAsync(order, order_in, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream)))
        return e;
    const Links L{bv.nodes, bv.leaf_parent, bv.root, seg_root, nullptr, nullptr};
    // the host vectors must outlive the copies above: run_levels synchronises
    return run_levels(c, A, L, order, (int32_t)tasks.size(), (int32_t)chunks.size(), (int32_t)blist.size());
}

size_t sah_top_bytes(int32_t nseg) {
    return 512 + sizeof(int32_t) * (size_t)nseg;   // counters | range | identity list
}

cudaError_t sah_top_prepare(rtsdf_ctx* c, void* scratch, int32_t nseg) {
    if (nseg < 1 || nseg > SAH_CH) return cudaErrorInvalidValue;
    std::vector<unsigned char> h(sah_top_bytes(nseg), 0);
    SahRange r{0, nseg, -1, 0};
    memcpy(h.data() + 256, &r, sizeof(r));
    int32_t* list = (int32_t*)(h.data() + 512);
    for (int32_t j = 0; j < nseg; j++) list[j] = j;
    cudaError_t e = cudaMemcpyAsync(scratch, h.data(), h.size(), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);   // h is a local buffer
    return e;
}

cudaError_t sah_top(rtsdf_ctx* c, void* scratch, int32_t nseg, const float4* boxes, const int32_t* node_ids,
                    const int32_t* child_of) {
    Bvh& bv = c->bvh;
    if (nseg < 1 || nseg > SAH_CH) return cudaErrorInvalidValue;
    if (nseg == 1) {
        RTSDF_LAUNCH(c, k_sah_top_single, 1, 1, 0, child_of, bv.nodes, bv.leaf_parent, bv.root);
        return cudaGetLastError();
    }
    cudaError_t e = block_attr(c);
    if (e) return e;
    unsigned char* p = (unsigned char*)scratch;
    int32_t* counters = (int32_t*)p;
    SahRange* range = (SahRange*)(p + 256);
    int32_t* list = (int32_t*)(p + 512);
    const Links L{bv.nodes, bv.leaf_parent, bv.root, nullptr, node_ids, child_of};
    // counters, the range {0, nseg} and the identity list come from sah_top_prepare
    RTSDF_LAUNCH(c, k_sah_block, 1, SAH_THREADS, sizeof(BlockSmem), range, list, list, boxes, (int32_t*)nullptr, L,
                 counters);
    return cudaGetLastError();
}

}  // namespace rtsdf
