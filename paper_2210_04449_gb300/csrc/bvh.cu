// Acceleration structure for the Sec. 2.2 closest-hit ray casts.
//
// The paper does not describe its ray-tracing structure.  This is a linear
// BVH: triangles ordered by the 30-bit Morton code of their centroid
// (stable LSD radix sort, so equal codes keep triangle order), the binary
// hierarchy of Karras ("Maximizing parallelism in the construction of BVHs,
// octrees and k-d trees", HPG 2012) over the unique keys (code, index), and
// child boxes filled bottom-up with one atomic counter per node.  A refit
// recomputes the leaf data and boxes for moved vertices with the same
// topology.  Leaf boxes are padded outward by 2^-16 extent (+ 2^-18 of the
// coordinate) so that fp32 rounding in the box test can never cull a
// triangle that the fp32 ray/triangle test would hit.
//
// Also here: the rigid per-object motion of animated scenes.
#include <math_constants.h>
#include <string.h>

#include <utility>
#include <vector>

#include "internal.cuh"

namespace rtsdf {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t nt,
                         float lx, float ly, float lz, float inv_w, uint32_t* __restrict__ keys,
                         int32_t* __restrict__ vals) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float c[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3; k++) {
        const float* p = verts + 3 * (int64_t)tris[3 * t + k];
        c[0] += p[0];
        c[1] += p[1];
        c[2] += p[2];
    }
    const float l[3] = {lx, ly, lz};
    uint32_t cell[3];
    for (int a = 0; a < 3; a++) {
        float u = (c[a] * (1.f / 3.f) - l[a]) * inv_w * 1024.f;
        u = fminf(fmaxf(u, 0.f), 1023.f);
        cell[a] = (uint32_t)u;
    }
    keys[t] = spread10(cell[0]) | (spread10(cell[1]) << 1) | (spread10(cell[2]) << 2);
    vals[t] = (int32_t)t;
}

__global__ void __launch_bounds__(SORT_THREADS) k_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                      uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; it++) {
        int64_t e = base + it * SORT_THREADS + threadIdx.x;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of `total` counters, one block of 1024 threads
__global__ void __launch_bounds__(1024) k_scan(uint32_t* __restrict__ a, int64_t total) {
    __shared__ uint32_t part[1024];
    const int64_t per = (total + 1023) / 1024;
    const int64_t lo = threadIdx.x * per, hi = min(lo + per, total);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; i++) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int64_t i = lo; i < hi; i++) {
        uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// stable scatter: element order inside a block is (item, warp, lane)
__global__ void __launch_bounds__(SORT_THREADS) k_scatter(const uint32_t* __restrict__ kin,
                                                         const int32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                         int64_t n, int shift, const uint32_t* __restrict__ hist,
                                                         int nblocks) {
    __shared__ uint32_t base[257];
    base[threadIdx.x] = hist[(size_t)threadIdx.x * nblocks + blockIdx.x];
    if (threadIdx.x == 0) base[256] = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t b0 = (int64_t)blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; it++) {
        const int64_t e = b0 + it * SORT_THREADS + threadIdx.x;
        const bool valid = e < n;
        uint32_t k = 0;
        int32_t v = 0;
        uint32_t d = 256;
        if (valid) {
            k = kin[e];
            v = vin[e];
            d = (k >> shift) & 0xFF;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & lt);
        const bool leader = (peers & lt) == 0;
        uint32_t pos = 0;
        for (unsigned w = 0; w < SORT_THREADS / 32; w++) {
            if (warp == w) {
                pos = base[d] + rank;
                __syncwarp();
                if (leader) base[d] += __popc(peers);
            }
            __syncthreads();
        }
        if (valid) {
            kout[pos] = k;
            vout[pos] = v;
        }
    }
}

__device__ __forceinline__ int delta(const uint32_t* __restrict__ mk, const int32_t* __restrict__ mv, int64_t n,
                                     int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const unsigned long long a = ((unsigned long long)mk[i] << 32) | (uint32_t)mv[i];
    const unsigned long long b = ((unsigned long long)mk[j] << 32) | (uint32_t)mv[j];
    return __clzll(a ^ b);
}

__global__ void k_karras(const uint32_t* __restrict__ mk, const int32_t* __restrict__ mv, int64_t n,
                         BNode* __restrict__ nodes, int32_t* __restrict__ leaf_parent) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(mk, mv, n, i, i + 1) - delta(mk, mv, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(mk, mv, n, i, i - d);
    int64_t lmax = 2;
    while (delta(mk, mv, n, i, i + lmax * d) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
        if (delta(mk, mv, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(mk, mv, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(mk, mv, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t g = i + s * d + min(d, 0);
    const int64_t lo = min(i, j), hi = max(i, j);
    int left, right;
    if (lo == g) { left = ~(int)g; leaf_parent[g] = (int)i; }
    else { left = (int)g; nodes[g].d.z = (int)i; }
    if (hi == g + 1) { right = ~(int)(g + 1); leaf_parent[g + 1] = (int)i; }
    else { right = (int)(g + 1); nodes[g + 1].d.z = (int)i; }
    nodes[i].d.x = left;
    nodes[i].d.y = right;
    if (i == 0) nodes[0].d.z = -1;
}

__device__ __forceinline__ float pad_lo(float v, float pad) { return v - (pad + fabsf(v) * 0x1p-18f); }
__device__ __forceinline__ float pad_hi(float v, float pad) { return v + (pad + fabsf(v) * 0x1p-18f); }

__device__ __forceinline__ void store_child(BNode* node, bool right, const float lo[3], const float hi[3]) {
    float* a = right ? &node->b.x : &node->a.x;
    a[0] = lo[0]; a[1] = hi[0]; a[2] = lo[1]; a[3] = hi[1];
    float* c = &node->c.x + (right ? 2 : 0);
    c[0] = lo[2]; c[1] = hi[2];
}

// Bottom-up boxes from `child` (a node id, or ~leaf) with box (lo, hi)
// whose parent is `node`: each node takes the box of its first-arriving
// child into its child slot and counts the arrival; the second arrival
// forms the union and climbs on.  A negative parent ends the climb.
__device__ __forceinline__ void climb(BNode* nodes, uint32_t* flags, float* __restrict__ nbox, int child, int node,
                                      float lo[3], float hi[3], int64_t guard_n) {
    // a tree over n leaves has depth < n; the guard only bounds the loop
    for (int64_t guard = 0; node >= 0 && guard < guard_n; guard++) {
        BNode* nd = nodes + node;
        const bool right = nd->d.y == child;
        store_child(nd, right, lo, hi);
        __threadfence();
        if (atomicAdd(flags + node, 1u) != 1u) return;   // first arrival: the sibling finishes this node
        __threadfence();
        // both children present: box of this node = union of its two child boxes
        const volatile float* a = &nd->a.x;
        const volatile float* b = &nd->b.x;
        const volatile float* c = &nd->c.x;
        lo[0] = fminf(a[0], b[0]); hi[0] = fmaxf(a[1], b[1]);
        lo[1] = fminf(a[2], b[2]); hi[1] = fmaxf(a[3], b[3]);
        lo[2] = fminf(c[0], c[2]); hi[2] = fmaxf(c[1], c[3]);
        for (int k = 0; k < 3; k++) {
            nbox[6 * (int64_t)node + k] = lo[k];
            nbox[6 * (int64_t)node + 3 + k] = hi[k];
        }
        child = node;
        node = nd->d.z;
    }
}

// Leaf data + bottom-up boxes.  One thread per leaf.
__global__ void k_leaves_up(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                            const int32_t* order, int64_t n, float4* __restrict__ tri, int32_t* leaf_tri,
                            const int32_t* __restrict__ leaf_parent, BNode* nodes, uint32_t* flags, float pad,
                            float* __restrict__ lbox, float* __restrict__ nbox) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = order[i];
    const float* p0 = verts + 3 * (int64_t)tris[3 * (int64_t)t];
    const float* p1 = verts + 3 * (int64_t)tris[3 * (int64_t)t + 1];
    const float* p2 = verts + 3 * (int64_t)tris[3 * (int64_t)t + 2];
    const float v0[3] = {p0[0], p0[1], p0[2]}, v1[3] = {p1[0], p1[1], p1[2]}, v2[3] = {p2[0], p2[1], p2[2]};
    tri[TRI_F4 * i + 0] = make_float4(v0[0], v0[1], v0[2], __int_as_float(t));
    tri[TRI_F4 * i + 1] = make_float4(__fsub_rn(v1[0], v0[0]), __fsub_rn(v1[1], v0[1]), __fsub_rn(v1[2], v0[2]), 0.f);
    tri[TRI_F4 * i + 2] = make_float4(__fsub_rn(v2[0], v0[0]), __fsub_rn(v2[1], v0[1]), __fsub_rn(v2[2], v0[2]), 0.f);
    tri[TRI_F4 * i + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
    leaf_tri[i] = t;
    if (n == 1) return;
    float lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = pad_lo(fminf(v0[a], fminf(v1[a], v2[a])), pad);
        hi[a] = pad_hi(fmaxf(v0[a], fmaxf(v1[a], v2[a])), pad);
        lbox[6 * i + a] = lo[a];
        lbox[6 * i + 3 + a] = hi[a];
    }
    climb(nodes, flags, nbox, ~(int)i, leaf_parent[i], lo, hi, n);
}

// ------------------------------------------------------- two-level form

// Object of each triangle (its first vertex's), and the identity order.
__global__ void k_tri_object(const int32_t* __restrict__ tris, const int32_t* __restrict__ vobj, int64_t n,
                             int n_obj, uint32_t* __restrict__ keys, int32_t* __restrict__ vals,
                             int32_t* __restrict__ count) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int o = min(max(vobj[tris[3 * t]], 0), n_obj - 1);
    keys[t] = (uint32_t)o;
    vals[t] = (int32_t)t;
    atomicAdd(count + o, 1);
}

// Cut the listed subtrees off the top tree, so that a refit climb stops at
// their roots.
__global__ void k_top_detach(const int32_t* __restrict__ child, int32_t n, BNode* nodes, int32_t* leaf_parent) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = child[j];
    if (c >= 0) nodes[c].d.z = -2;
    else leaf_parent[~c] = -2;
}

// Box of each listed subtree (its root's box) for the top-tree build.
__global__ void k_top_boxes(const int32_t* __restrict__ child, int32_t n, const float* __restrict__ nbox,
                            const float* __restrict__ lbox, float4* __restrict__ box) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = child[j];
    const float* p = c >= 0 ? nbox + 6 * (int64_t)c : lbox + 6 * (int64_t)(~c);
    box[2 * j] = make_float4(p[0], p[1], p[2], 0.f);
    box[2 * j + 1] = make_float4(p[3], p[4], p[5], 0.f);
}

// Boxes of the top tree: climb from every listed subtree root.
__global__ void k_top_up(const int32_t* __restrict__ child, int32_t n, const int32_t* __restrict__ leaf_parent,
                         BNode* nodes, uint32_t* flags, const float* __restrict__ lbox, float* __restrict__ nbox,
                         int64_t nt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = child[j];
    const float* p = c >= 0 ? nbox + 6 * (int64_t)c : lbox + 6 * (int64_t)(~c);
    float lo[3] = {p[0], p[1], p[2]}, hi[3] = {p[3], p[4], p[5]};
    climb(nodes, flags, nbox, c, c >= 0 ? nodes[c].d.z : leaf_parent[~c], lo, hi, nt);
}

// Child boxes of the 4-wide nodes from the (re)fitted binary boxes.
__global__ void k_wide_boxes(WNode* __restrict__ wide, int64_t n_wide, const float* __restrict__ nbox,
                             const float* __restrict__ lbox) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_wide * 4) return;
    const int64_t w = i >> 2;
    const int k = (int)(i & 3);
    const int src = (&wide[w].src.x)[k];
    float b[6] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
    if (src != WIDE_EMPTY) {
        const float* p = src >= 0 ? nbox + 6 * (int64_t)src : lbox + 6 * (int64_t)(~src);
        for (int a = 0; a < 6; a++) b[a] = p[a];
    }
    (&wide[w].lox.x)[k] = b[0];
    (&wide[w].hix.x)[k] = b[3];
    (&wide[w].loy.x)[k] = b[1];
    (&wide[w].hiy.x)[k] = b[4];
    (&wide[w].loz.x)[k] = b[2];
    (&wide[w].hiz.x)[k] = b[5];
}

__global__ void k_depth(const int32_t* __restrict__ leaf_parent, const BNode* __restrict__ nodes, int64_t n,
                        int32_t* depth) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = 1;
    int node = n > 1 ? leaf_parent[i] : -1;
    while (node >= 0 && d < 4096) {
        d++;
        node = nodes[node].d.z;
    }
    atomicMax(depth, d);
}

// ---------------------------------------------------------------- motion
__global__ void k_obj_boxes_init(float* boxes, int n_obj) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_obj) return;
    for (int a = 0; a < 3; a++) {
        boxes[6 * i + a] = CUDART_INF_F;
        boxes[6 * i + 3 + a] = -CUDART_INF_F;
    }
}

__device__ __forceinline__ void atomic_min_f(float* a, float v) {
    if (v >= 0.f) atomicMin(reinterpret_cast<int*>(a), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float* a, float v) {
    if (v >= 0.f) atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));
    else atomicMin(reinterpret_cast<unsigned*>(a), __float_as_uint(v));
}

// Box of every moved object (before the move), then v += t[obj].
__global__ void k_obj_boxes(const float* __restrict__ verts, const int32_t* __restrict__ vobj, int64_t nv,
                            const float* __restrict__ trans, float* boxes) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int o = vobj[i];
    const float* t = trans + 3 * o;
    if (t[0] == 0.f && t[1] == 0.f && t[2] == 0.f) return;
    for (int a = 0; a < 3; a++) {
        atomic_min_f(boxes + 6 * o + a, verts[3 * i + a]);
        atomic_max_f(boxes + 6 * o + 3 + a, verts[3 * i + a]);
    }
}

__global__ void k_moved_list(const float* __restrict__ trans, int n_obj, int32_t* list, int32_t* count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_obj) return;
    const float* t = trans + 3 * i;
    if (t[0] != 0.f || t[1] != 0.f || t[2] != 0.f) list[atomicAdd(count, 1)] = i;
}

__global__ void k_translate(float* __restrict__ verts, const int32_t* __restrict__ vobj, int64_t nv,
                            const float* __restrict__ trans) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv * 3) return;
    const int64_t v = i / 3;
    const int a = (int)(i % 3);
    verts[i] = __fadd_rn(verts[i], trans[3 * vobj[v] + a]);
}

// Rigid transforms, rows of [R | t] per object (12 floats).  An object is
// moved unless its transform is exactly the identity.
__device__ __forceinline__ bool xform_moves(const float* m) {
    return m[0] != 1.f || m[1] != 0.f || m[2] != 0.f || m[3] != 0.f || m[4] != 0.f || m[5] != 1.f ||
           m[6] != 0.f || m[7] != 0.f || m[8] != 0.f || m[9] != 0.f || m[10] != 1.f || m[11] != 0.f;
}

__global__ void k_moved_list_x(const float* __restrict__ xf, int n_obj, int32_t* list, int32_t* count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_obj) return;
    if (xform_moves(xf + 12 * i)) list[atomicAdd(count, 1)] = i;
}

// Box of every moved object before the transform.
__global__ void k_obj_boxes_x(const float* __restrict__ verts, const int32_t* __restrict__ vobj, int64_t nv,
                              const float* __restrict__ xf, float* boxes) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int o = vobj[i];
    if (!xform_moves(xf + 12 * o)) return;
    for (int a = 0; a < 3; a++) {
        atomic_min_f(boxes + 6 * o + a, verts[3 * i + a]);
        atomic_max_f(boxes + 6 * o + 3 + a, verts[3 * i + a]);
    }
}

// v' = R v + t in fp32, each product and sum rounded in this order:
// v'_a = ((R_a0 x + R_a1 y) + R_a2 z) + t_a  (no fused multiply-add).
__global__ void k_transform(float* __restrict__ verts, const int32_t* __restrict__ vobj, int64_t nv,
                            const float* __restrict__ xf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const float* m = xf + 12 * vobj[i];
    const float x = verts[3 * i], y = verts[3 * i + 1], z = verts[3 * i + 2];
    float out[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float* r = m + 4 * a;
        out[a] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[0], x), __fmul_rn(r[1], y)), __fmul_rn(r[2], z)), r[3]);
    }
    verts[3 * i] = out[0];
    verts[3 * i + 1] = out[1];
    verts[3 * i + 2] = out[2];
}

}  // namespace

// Collapse the binary tree into 4-wide nodes, on the device, one tree level
// at a time: every frontier node (a binary node that roots a wide node)
// starts from its two children and replaces the internal child of largest
// surface area by its two children until four are collected (or only
// leaves remain); each internal child roots a wide node of the next level.
// Slots are handed out in frontier order by an exclusive scan of the
// internal-child counts, so the layout is breadth-first with the children
// of a node contiguous.
namespace {

__device__ __forceinline__ float half_area(const float* __restrict__ nbox, int node) {
    const float* p = nbox + 6 * (int64_t)node;
    const float dx = p[3] - p[0], dy = p[4] - p[1], dz = p[5] - p[2];
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_collapse_expand(const int32_t* __restrict__ fb, int32_t cnt, const BNode* __restrict__ bn,
                                  const float* __restrict__ nbox, int4* __restrict__ kids,
                                  uint32_t* __restrict__ nint) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int4 d = bn[fb[i]].d;
    int kid[4] = {d.x, d.y, WIDE_EMPTY, WIDE_EMPTY};
    int nk = 2;
    while (nk < 4) {
        int best = -1;
        float ba = -1.f;
        for (int k = 0; k < nk; k++)
            if (kid[k] >= 0) {
                const float ar = half_area(nbox, kid[k]);
                if (ar > ba) {
                    ba = ar;
                    best = k;
                }
            }
        if (best < 0) break;
        const int4 od = bn[kid[best]].d;
        kid[best] = od.x;
        kid[nk++] = od.y;
    }
    kids[i] = make_int4(kid[0], kid[1], kid[2], kid[3]);
    nint[i] = (kid[0] >= 0) + (kid[1] >= 0) + (kid[2] >= 0) + (kid[3] >= 0);
}

__global__ void k_collapse_write(const int32_t* __restrict__ fslot, int32_t cnt, const int4* __restrict__ kids,
                                 const uint32_t* __restrict__ off, int32_t base, int64_t cap, WNode* __restrict__ wide,
                                 int32_t* __restrict__ nb, int32_t* __restrict__ nslot, int32_t* __restrict__ total) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int4 kv = kids[i];
    const int kid[4] = {kv.x, kv.y, kv.z, kv.w};
    const uint32_t o = off[i];
    uint32_t j = 0;
    int child[4], src[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        src[k] = kid[k];
        if (kid[k] == WIDE_EMPTY) {
            child[k] = WIDE_EMPTY;
        } else if (kid[k] >= 0) {
            const int32_t slot = base + (int32_t)(o + j);
            if ((int64_t)slot >= cap) {   // only a damaged tree gets here: drop the child, the host stops
                child[k] = src[k] = WIDE_EMPTY;
                j++;
                continue;
            }
            child[k] = slot;
            nb[o + j] = kid[k];
            nslot[o + j] = slot;
            j++;
        } else {
            child[k] = kid[k];   // ~leaf
        }
    }
    const int32_t w = fslot[i];
    wide[w].child = make_int4(child[0], child[1], child[2], child[3]);
    wide[w].src = make_int4(src[0], src[1], src[2], src[3]);
    if (i == cnt - 1) *total = (int32_t)(o + j);
}

__global__ void k_collapse_root(const int32_t* root, int32_t* fb, int32_t* fslot) {
    fb[0] = *root;
    fslot[0] = 0;
}

}  // namespace

static cudaError_t collapse_wide(rtsdf_ctx* c) {
    Bvh& b = c->bvh;
    const int64_t n = b.nt;                  // n >= 2: n - 1 binary internal nodes
    const int64_t cap = n - 1;               // every wide node roots a distinct binary node
    cudaError_t e;
    if (b.col_cap < cap) {
        cudaFree(b.col_fb); cudaFree(b.col_fslot); cudaFree(b.col_nb); cudaFree(b.col_nslot);
        cudaFree(b.col_kids); cudaFree(b.col_nint); cudaFree(b.col_total);
        b.col_fb = b.col_fslot = b.col_nb = b.col_nslot = b.col_total = nullptr;
        b.col_kids = nullptr;
        b.col_nint = nullptr;
        b.col_cap = 0;
        if ((e = cudaMalloc(&b.col_fb, sizeof(int32_t) * cap)) || (e = cudaMalloc(&b.col_fslot, sizeof(int32_t) * cap)) ||
            (e = cudaMalloc(&b.col_nb, sizeof(int32_t) * cap)) || (e = cudaMalloc(&b.col_nslot, sizeof(int32_t) * cap)) ||
            (e = cudaMalloc(&b.col_kids, sizeof(int4) * cap)) || (e = cudaMalloc(&b.col_nint, sizeof(uint32_t) * cap)) ||
            (e = cudaMalloc(&b.col_total, sizeof(int32_t))))
            return e;
        b.col_cap = cap;
    }
    if (b.wide_cap < cap) {
        // the texture over the old array may still be in use by a launch
        if ((e = cudaStreamSynchronize(c->stream))) return e;
        drop_texture(b.wtex);
        if (b.wide) cudaFree(b.wide);
        b.wide = nullptr;
        b.wide_cap = 0;
        if ((e = cudaMalloc(&b.wide, sizeof(WNode) * cap))) return e;
        b.wide_cap = cap;
        b.wtex = make_int4_texture(b.wide, (sizeof(WNode) / 16) * (size_t)cap, c->device);
    }
    int32_t *fb = b.col_fb, *fs = b.col_fslot, *nb = b.col_nb, *ns = b.col_nslot;
    RTSDF_LAUNCH(c, k_collapse_root, 1, 1, 0, b.root, fb, fs);
    int32_t base = 1, cnt = 1;
    while (cnt > 0) {
        const unsigned g = (unsigned)((cnt + 255) / 256);
        RTSDF_LAUNCH(c, k_collapse_expand, g, 256, 0, fb, cnt, b.nodes, b.nbox, b.col_kids, b.col_nint);
        RTSDF_LAUNCH(c, k_scan, 1, 1024, 0, b.col_nint, (int64_t)cnt);
        RTSDF_LAUNCH(c, k_collapse_write, g, 256, 0, fs, cnt, b.col_kids, b.col_nint, base, cap, b.wide, nb, ns,
                     b.col_total);
        int32_t next = 0;
        e = cudaMemcpyAsync(&next, b.col_total, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        if (next < 0 || (int64_t)base + next > cap) return cudaErrorUnknown;   // only a damaged tree gets here
        base += next;
        cnt = next;
        int32_t* t = fb; fb = nb; nb = t;
        t = fs; fs = ns; ns = t;
    }
    b.n_wide = base;
    RTSDF_LAUNCH(c, k_wide_boxes, (unsigned)((4 * b.n_wide + 255) / 256), 256, 0, b.wide, b.n_wide, b.nbox, b.lbox);
    return cudaGetLastError();
}

// Two-level topology: triangles sorted by object (stable), one SAH subtree
// per object, and the top tree over the objects' subtrees.  Sets *order to
// the leaf order.  *applies = false (nothing built) when the form does not
// apply: no objects, or more than SAH_TOP_MAX objects with triangles.
static cudaError_t two_level_topology(rtsdf_ctx* c, int32_t** order, bool* applies) {
    Bvh& b = c->bvh;
    const int64_t n = b.nt;
    const int n_obj = c->n_obj;
    *applies = false;
    b.two_level = false;
    if (n < 2 || n_obj < 1 || !c->vert_obj) return cudaSuccess;
    cudaError_t e;
    if (b.obj_cap < n_obj) {
        cudaFree(b.obj_count);
        b.obj_count = nullptr;
        b.obj_cap = 0;
        if ((e = cudaMalloc(&b.obj_count, sizeof(int32_t) * (size_t)n_obj))) return e;
        b.obj_cap = n_obj;
    }
    const unsigned g = (unsigned)((n + 255) / 256);
    const int nblocks = (int)((n + SORT_TILE - 1) / SORT_TILE);
    if ((e = cudaMemsetAsync(b.obj_count, 0, sizeof(int32_t) * (size_t)n_obj, c->stream))) return e;
    RTSDF_LAUNCH(c, k_tri_object, g, 256, 0, c->tris, c->vert_obj, n, n_obj, b.mk0, b.mv0, b.obj_count);
    int bits = 1;
    while (bits < 32 && (1u << bits) < (unsigned)n_obj) bits++;
    uint32_t* kin = b.mk0; uint32_t* kout = b.mk1;
    int32_t* vin = b.mv0; int32_t* vout = b.mv1;
    for (int shift = 0; shift < bits; shift += 8) {
        RTSDF_LAUNCH(c, k_hist, nblocks, SORT_THREADS, 0, kin, n, shift, b.hist, nblocks);
        RTSDF_LAUNCH(c, k_scan, 1, 1024, 0, b.hist, (int64_t)256 * nblocks);
        RTSDF_LAUNCH(c, k_scatter, nblocks, SORT_THREADS, 0, kin, vin, kout, vout, n, shift, b.hist, nblocks);
        uint32_t* tk = kin; kin = kout; kout = tk;
        int32_t* tv = vin; vin = vout; vout = tv;
    }
    std::vector<int32_t> count((size_t)n_obj);
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaMemcpyAsync(count.data(), b.obj_count, sizeof(int32_t) * (size_t)n_obj, cudaMemcpyDeviceToHost,
                             c->stream)))
        return e;
    if ((e = cudaStreamSynchronize(c->stream))) return e;
    std::vector<int32_t> bounds(1, 0);
    for (int o = 0; o < n_obj; o++)
        if (count[(size_t)o] > 0) bounds.push_back(bounds.back() + count[(size_t)o]);
    const int32_t k = (int32_t)bounds.size() - 1;
    if (k < 1 || k > SAH_TOP_MAX || bounds.back() != n) return cudaSuccess;
    if (b.top_cap < k) {
        cudaFree(b.top_child); cudaFree(b.top_ids); cudaFree(b.top_box); cudaFree(b.top_scratch);
        b.top_child = b.top_ids = nullptr;
        b.top_box = nullptr;
        b.top_scratch = nullptr;
        b.top_cap = 0;
        if ((e = cudaMalloc(&b.top_child, sizeof(int32_t) * (size_t)k)) ||
            (e = cudaMalloc(&b.top_ids, sizeof(int32_t) * (size_t)k)) ||
            (e = cudaMalloc(&b.top_box, sizeof(float4) * 2 * (size_t)k)) ||
            (e = cudaMalloc(&b.top_scratch, sah_top_bytes(SAH_TOP_MAX))))
            return e;
        b.top_cap = k;
    }
    // leaves of one-triangle objects keep parent -1 until the top tree takes them
    if ((e = cudaMemsetAsync(b.leaf_parent, 0xFF, sizeof(int32_t) * (size_t)n, c->stream))) return e;
    int32_t* out = vin == b.mv0 ? b.mv1 : b.mv0;
    if ((e = sah_segments(c, b.sah, out, vin, bounds.data(), k, b.top_child))) return e;
    // the top tree's nodes own the boundaries between objects
    std::vector<int32_t> ids((size_t)k, 0);
    for (int32_t j = 0; j + 1 < k; j++) ids[(size_t)j] = bounds[(size_t)j + 1] - 1;
    if ((e = cudaMemcpyAsync(b.top_ids, ids.data(), sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, c->stream)))
        return e;
    if ((e = sah_top_prepare(c, b.top_scratch, k))) return e;   // synchronises: ids may go
    b.top_n = k;
    b.two_level = true;
    *applies = true;
    *order = out;
    return cudaSuccess;
}

// Top tree of the two-level form over its subtrees, whose boxes are fitted
// (flags of the top nodes zero), then the top boxes.
static cudaError_t build_top(rtsdf_ctx* c) {
    Bvh& b = c->bvh;
    const unsigned gk = (unsigned)((b.top_n + 127) / 128);
    RTSDF_LAUNCH(c, k_top_boxes, gk, 128, 0, b.top_child, b.top_n, b.nbox, b.lbox, b.top_box);
    cudaError_t e = sah_top(c, b.top_scratch, b.top_n, b.top_box, b.top_ids, b.top_child);
    if (e) return e;
    RTSDF_LAUNCH(c, k_top_up, gk, 128, 0, b.top_child, b.top_n, b.leaf_parent, b.nodes, b.flags, b.lbox, b.nbox,
                 b.nt);
    return cudaGetLastError();
}

cudaError_t launch_bvh_build(rtsdf_ctx* c) {
    Bvh& b = c->bvh;
    const int64_t n = c->nt;
    b.nt = n;
    b.built = false;
    b.n_wide = 0;
    if (n == 0) {
        b.depth = 0;
        b.built = true;
        return cudaSuccess;
    }
    cudaError_t e;
    // the two-level form falls back to one SAH tree where it does not apply
    const bool sah = c->bvh_builder != RTSDF_BVH_LBVH && n > 1;
    const int nblocks = (int)((n + SORT_TILE - 1) / SORT_TILE);
    // per-triangle arrays and scratch grow with the mesh and are kept across
    // builds, so a per-frame rebuild allocates nothing
    if (b.cap_nt < n) {
        cudaFree(b.nodes); cudaFree(b.tri); cudaFree(b.leaf_tri); cudaFree(b.leaf_parent); cudaFree(b.flags);
        cudaFree(b.lbox); cudaFree(b.nbox); cudaFree(b.mk0); cudaFree(b.mk1); cudaFree(b.mv0); cudaFree(b.mv1);
        cudaFree(b.hist);
        b.nodes = nullptr; b.tri = nullptr; b.leaf_tri = b.leaf_parent = nullptr; b.flags = nullptr;
        b.lbox = b.nbox = nullptr; b.mk0 = b.mk1 = b.hist = nullptr; b.mv0 = b.mv1 = nullptr;
        b.cap_nt = 0;
        const size_t nn = (size_t)n;
        if ((e = cudaMalloc(&b.nodes, sizeof(BNode) * (nn > 1 ? nn - 1 : 1))) ||
            (e = cudaMalloc(&b.tri, sizeof(float4) * TRI_F4 * nn)) ||
            (e = cudaMalloc(&b.leaf_tri, sizeof(int32_t) * nn)) ||
            (e = cudaMalloc(&b.leaf_parent, sizeof(int32_t) * nn)) ||
            (e = cudaMalloc(&b.flags, sizeof(uint32_t) * nn)) || (e = cudaMalloc(&b.lbox, sizeof(float) * 6 * nn)) ||
            (e = cudaMalloc(&b.nbox, sizeof(float) * 6 * (nn > 1 ? nn - 1 : 1))) ||
            (e = cudaMalloc(&b.mk0, sizeof(uint32_t) * nn)) || (e = cudaMalloc(&b.mk1, sizeof(uint32_t) * nn)) ||
            (e = cudaMalloc(&b.mv0, sizeof(int32_t) * nn)) || (e = cudaMalloc(&b.mv1, sizeof(int32_t) * nn)) ||
            (e = cudaMalloc(&b.hist, sizeof(uint32_t) * 256 * (size_t)nblocks)))
            return e;
        b.cap_nt = n;
    }
    if (!b.root && (e = cudaMalloc(&b.root, sizeof(int32_t)))) return e;
    if (!b.d_depth && (e = cudaMalloc(&b.d_depth, sizeof(int32_t)))) return e;
    if (sah && b.sah_bytes < sah_scratch_bytes(n)) {
        cudaFree(b.sah);
        b.sah = nullptr;
        b.sah_bytes = 0;
        if ((e = cudaMalloc(&b.sah, sah_scratch_bytes(n)))) return e;
        b.sah_bytes = sah_scratch_bytes(n);
    }
    const unsigned g = (unsigned)((n + 255) / 256);
    int32_t* order = b.mv0;                    // triangle at each leaf position
    bool two = false;
    if (c->bvh_builder == RTSDF_BVH_TWO_LEVEL && (e = two_level_topology(c, &order, &two))) return e;
    if (two) {
        // topology below the top tree done; the top tree follows the boxes
    } else if (sah) {
        if ((e = sah_topology(c, b.sah, order))) return e;
    } else {
        const float w = 2.f * c->cfg.extent;
        const float lx = c->cfg.bmin[0] - 0.5f * c->cfg.extent, ly = c->cfg.bmin[1] - 0.5f * c->cfg.extent,
                    lz = c->cfg.bmin[2] - 0.5f * c->cfg.extent;
        RTSDF_LAUNCH(c, k_morton, g, 256, 0, c->verts, c->tris, n, lx, ly, lz, 1.f / w, b.mk0, b.mv0);
        uint32_t* kin = b.mk0; uint32_t* kout = b.mk1;
        int32_t* vin = b.mv0; int32_t* vout = b.mv1;
        for (int shift = 0; shift < 32; shift += 8) {
            RTSDF_LAUNCH(c, k_hist, nblocks, SORT_THREADS, 0, kin, n, shift, b.hist, nblocks);
            RTSDF_LAUNCH(c, k_scan, 1, 1024, 0, b.hist, (int64_t)256 * nblocks);
            RTSDF_LAUNCH(c, k_scatter, nblocks, SORT_THREADS, 0, kin, vin, kout, vout, n, shift, b.hist, nblocks);
            uint32_t* tk = kin; kin = kout; kout = tk;
            int32_t* tv = vin; vin = vout; vout = tv;
        }
        // four passes: sorted keys back in mk0, triangle order in mv0
        order = vin;
        if ((e = cudaMemsetAsync(b.root, 0, sizeof(int32_t), c->stream))) return e;
        if (n > 1)
            RTSDF_LAUNCH(c, k_karras, (unsigned)((n - 1 + 255) / 256), 256, 0, kin, vin, n, b.nodes, b.leaf_parent);
    }
    if ((e = cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, c->stream))) return e;
    const float pad = c->cfg.extent * 0x1p-16f;
    RTSDF_LAUNCH(c, k_leaves_up, g, 256, 0, c->verts, c->tris, order, n, b.tri, b.leaf_tri, b.leaf_parent, b.nodes,
                 b.flags, pad, b.lbox, b.nbox);
    if (two && (e = build_top(c))) return e;
    if ((e = cudaMemsetAsync(b.d_depth, 0, sizeof(int32_t), c->stream))) return e;
    RTSDF_LAUNCH(c, k_depth, g, 256, 0, b.leaf_parent, b.nodes, n, b.d_depth);
    if (n > 1) {
        if ((e = cudaGetLastError())) return e;
        if ((e = collapse_wide(c))) return e;
    }
    if ((e = cudaGetLastError())) return e;
    int32_t hd = 0;
    if ((e = cudaMemcpyAsync(&hd, b.d_depth, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream))) return e;
    if ((e = cudaStreamSynchronize(c->stream))) return e;
    b.depth = hd;
    b.built = true;
    return cudaSuccess;
}

cudaError_t launch_bvh_refit(rtsdf_ctx* c) {
    Bvh& b = c->bvh;
    const int64_t n = b.nt;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, c->stream);
    if (e != cudaSuccess) return e;
    const float pad = c->cfg.extent * 0x1p-16f;
    if (b.two_level) {
        // refit the objects' subtrees, then rebuild the top tree over them
        RTSDF_LAUNCH(c, k_top_detach, (unsigned)((b.top_n + 127) / 128), 128, 0, b.top_child, b.top_n, b.nodes,
                     b.leaf_parent);
        RTSDF_LAUNCH(c, k_leaves_up, (unsigned)((n + 255) / 256), 256, 0, c->verts, c->tris, b.leaf_tri, n, b.tri,
                     b.leaf_tri, b.leaf_parent, b.nodes, b.flags, pad, b.lbox, b.nbox);
        if ((e = build_top(c))) return e;
        return collapse_wide(c);
    }
    RTSDF_LAUNCH(c, k_leaves_up, (unsigned)((n + 255) / 256), 256, 0, c->verts, c->tris, b.leaf_tri, n, b.tri,
                 b.leaf_tri, b.leaf_parent, b.nodes, b.flags, pad, b.lbox, b.nbox);
    if (b.n_wide > 0)
        RTSDF_LAUNCH(c, k_wide_boxes, (unsigned)((4 * b.n_wide + 255) / 256), 256, 0, b.wide, b.n_wide, b.nbox, b.lbox);
    return cudaGetLastError();
}

cudaError_t launch_move(rtsdf_ctx* c) {
    const int n_obj = c->n_obj;
    cudaError_t e = cudaMemsetAsync(c->d_moved_count, 0, sizeof(int32_t), c->stream);
    if (e != cudaSuccess) return e;
    RTSDF_LAUNCH(c, k_obj_boxes_init, (n_obj + 127) / 128, 128, 0, c->obj_box, n_obj);
    RTSDF_LAUNCH(c, k_moved_list, (n_obj + 127) / 128, 128, 0, c->obj_trans, n_obj, c->moved_list, c->d_moved_count);
    if (c->nv > 0) {
        RTSDF_LAUNCH(c, k_obj_boxes, (unsigned)((c->nv + 255) / 256), 256, 0, c->verts, c->vert_obj, c->nv,
                     c->obj_trans, c->obj_box);
        RTSDF_LAUNCH(c, k_translate, (unsigned)((c->nv * 3 + 255) / 256), 256, 0, c->verts, c->vert_obj, c->nv,
                     c->obj_trans);
    }
    return cudaGetLastError();
}

cudaError_t launch_transform(rtsdf_ctx* c) {
    const int n_obj = c->n_obj;
    cudaError_t e = cudaMemsetAsync(c->d_moved_count, 0, sizeof(int32_t), c->stream);
    if (e != cudaSuccess) return e;
    RTSDF_LAUNCH(c, k_obj_boxes_init, (n_obj + 127) / 128, 128, 0, c->obj_box, n_obj);
    RTSDF_LAUNCH(c, k_moved_list_x, (n_obj + 127) / 128, 128, 0, c->obj_xform, n_obj, c->moved_list,
                 c->d_moved_count);
    if (c->nv > 0) {
        RTSDF_LAUNCH(c, k_obj_boxes_x, (unsigned)((c->nv + 255) / 256), 256, 0, c->verts, c->vert_obj, c->nv,
                     c->obj_xform, c->obj_box);
        RTSDF_LAUNCH(c, k_transform, (unsigned)((c->nv + 255) / 256), 256, 0, c->verts, c->vert_obj, c->nv,
                     c->obj_xform);
    }
    return cudaGetLastError();
}

cudaTextureObject_t make_int4_texture(const void* ptr, size_t count, int device) {
    int maxw = 0;
    if (!ptr || count == 0 || cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, device) != cudaSuccess ||
        count > (size_t)maxw)
        return 0;
    cudaResourceDesc rd;
    memset(&rd, 0, sizeof(rd));
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = const_cast<void*>(ptr);
    rd.res.linear.desc = cudaCreateChannelDesc<int4>();
    rd.res.linear.sizeInBytes = count * sizeof(int4);
    cudaTextureDesc td;
    memset(&td, 0, sizeof(td));
    td.readMode = cudaReadModeElementType;
    cudaTextureObject_t t = 0;
    if (cudaCreateTextureObject(&t, &rd, &td, nullptr) != cudaSuccess) {
        (void)cudaGetLastError();   // a failed creation leaves no error behind: plain loads serve
        return 0;
    }
    return t;
}

void drop_texture(cudaTextureObject_t& t) {
    if (t) cudaDestroyTextureObject(t);
    t = 0;
}

}  // namespace rtsdf
