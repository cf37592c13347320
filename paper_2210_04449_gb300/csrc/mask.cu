// Sec. 2.2 / Eq. 1 -- near-surface mask, coarse fill and accumulator upkeep.
//
// A fine texel is traced iff the coarse SDF at its parent voxel satisfies
// c_t <= d (Eq. 1, first case).  With c = h_c (sqrt(D2) - beta) and integer
// D2 this is exactly D2 <= T, T = floor((d + beta)^2) (d, beta in coarse
// voxels), so the mask is an integer decision.  All 8 fine children of a
// coarse voxel share its decision, so one thread handles one coarse voxel:
//   * unmasked: f = c for the 8 children (Eq. 1, second case); a child with
//     an accumulated distance restarts (u = +inf, counts = 0);
//   * masked: the voxel is appended to the trace list; each child may be
//     reset (a moved object's previous box lies within u of its centre),
//     then u <- alpha u + (1 - alpha) c (Eq. 1's decay; the minimum with the
//     new rays is taken by the tracer).
#include <math_constants.h>

#include <math.h>

#include "internal.cuh"

namespace rtsdf {

int64_t mask_threshold(float d_vox, float beta_vox) {
    double s = (double)d_vox + (double)beta_vox;
    if (s < 0) return -1;
    return (int64_t)floor(s * s);
}

namespace {

// fp32, fixed order: d = max(max(lo - p, p - hi), 0); d2 = (dx dx + dy dy) + dz dz
__device__ __forceinline__ bool within(const float* __restrict__ b, float px, float py, float pz, float uu) {
    const float dx = fmaxf(fmaxf(__fsub_rn(b[0], px), __fsub_rn(px, b[3])), 0.f);
    const float dy = fmaxf(fmaxf(__fsub_rn(b[1], py), __fsub_rn(py, b[4])), 0.f);
    const float dz = fmaxf(fmaxf(__fsub_rn(b[2], pz), __fsub_rn(pz, b[5])), 0.f);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return d2 <= uu;
}

// Moved boxes are binned into cells of BIN_VOX^3 coarse voxels, each box
// dilated by BIN_REACH coarse voxels (+1 cell of slack against rounding).
// A texel whose accumulated distance u is at most BIN_REACH voxels can only
// be within u of boxes listed in its own cell; other texels test every
// moved box.  Both paths apply the same fp32 test, so the result equals the
// test against all moved boxes.
constexpr int BIN_VOX = 8;
constexpr float BIN_REACH = 4.f;

struct BinArgs {
    const float* boxes;
    const int32_t* moved;
    const int32_t* n_moved;
    int g;                 // cells per axis
    float bx, by, bz, inv_cell, reach;
    uint32_t* count;       // [g^3]
    uint32_t* start;       // [g^3 + 1]
    uint32_t* cursor;      // [g^3]
    int32_t* items;
    uint32_t cap;
    uint32_t* overflow;
};

__device__ __forceinline__ void box_cells(const BinArgs& a, const float* b, int lo[3], int hi[3]) {
    const float o[3] = {a.bx, a.by, a.bz};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        lo[k] = max((int)floorf((b[k] - a.reach - o[k]) * a.inv_cell) - 1, 0);
        hi[k] = min((int)floorf((b[3 + k] + a.reach - o[k]) * a.inv_cell) + 1, a.g - 1);
    }
}

// One warp per moved object; its lanes share the object's range of cells.
__device__ __forceinline__ int box_cell_range(const BinArgs& a, const float* b, int lo[3], int n[3]) {
    int hi[3];
    box_cells(a, b, lo, hi);
    for (int k = 0; k < 3; k++) n[k] = hi[k] >= lo[k] ? hi[k] - lo[k] + 1 : 0;
    return n[0] * n[1] * n[2];
}

__global__ void k_bin_count(BinArgs a) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = (int)(threadIdx.x & 31);
    if (w >= *a.n_moved) return;
    int lo[3], n[3];
    const int total = box_cell_range(a, a.boxes + 6 * a.moved[w], lo, n);
    for (int i = lane; i < total; i += 32) {
        const int x = lo[0] + i % n[0], y = lo[1] + (i / n[0]) % n[1], z = lo[2] + i / (n[0] * n[1]);
        atomicAdd(a.count + x + a.g * (y + a.g * z), 1u);
    }
}

// exclusive scan of the cell counts (one block, 1024 cells per round,
// coalesced); start[g^3] = total
__global__ void __launch_bounds__(1024) k_bin_scan(BinArgs a) {
    __shared__ uint32_t wsum[32];
    const int64_t total = (int64_t)a.g * a.g * a.g;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int64_t base = 0; base < total; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < total ? a.count[i] : 0u;
        uint32_t x = v;   // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if ((int)lane >= o) w += y;
            }
            wsum[lane] = w;   // inclusive over the warps
        }
        __syncthreads();
        if (i < total) {
            a.start[i] = carry + (warp ? wsum[warp - 1] : 0u) + x - v;
            a.cursor[i] = 0;
        }
        carry += wsum[31];
        __syncthreads();   // wsum is rewritten next round
    }
    if (threadIdx.x == 0) {
        a.start[total] = carry;
        if (carry > a.cap) *a.overflow = 1u;
    }
}

__global__ void k_bin_fill(BinArgs a) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = (int)(threadIdx.x & 31);
    if (w >= *a.n_moved || *a.overflow) return;
    const int obj = a.moved[w];
    int lo[3], n[3];
    const int total = box_cell_range(a, a.boxes + 6 * obj, lo, n);
    for (int i = lane; i < total; i += 32) {
        const int x = lo[0] + i % n[0], y = lo[1] + (i / n[0]) % n[1], z = lo[2] + i / (n[0] * n[1]);
        const int c = x + a.g * (y + a.g * z);
        a.items[a.start[c] + atomicAdd(a.cursor + c, 1u)] = obj;
    }
}

struct MaskArgs {
    const uint32_t* seeds;
    const float* coarse;
    int nc;
    long long T;
    float* accum;
    uint32_t* counts;
    float* fine;
    uint32_t* list;
    uint32_t* count;
    float alpha;
    // reset in changed regions
    const float* boxes;
    const int32_t* moved;
    const int32_t* n_moved;
    int reset;
    float bx, by, bz, hf;
    // binned moved boxes
    const uint32_t* bin_start;
    const int32_t* bin_items;
    const uint32_t* bin_overflow;
    int bin_g;
    float reach;   // BIN_REACH coarse voxels in world units
};

__device__ __forceinline__ bool near_moved_box(const MaskArgs& a, int cx, int cy, int cz, float px, float py,
                                               float pz, float u, int n_moved) {
    const float uu = __fmul_rn(u, u);
    if (u <= a.reach && !*a.bin_overflow) {
        const int c = cx / BIN_VOX + a.bin_g * (cy / BIN_VOX + a.bin_g * (cz / BIN_VOX));
        const uint32_t e = a.bin_start[c + 1];
        for (uint32_t i = a.bin_start[c]; i < e; i++)
            if (within(a.boxes + 6 * a.bin_items[i], px, py, pz, uu)) return true;
        return false;
    }
    for (int i = 0; i < n_moved; i++)
        if (within(a.boxes + 6 * a.moved[i], px, py, pz, uu)) return true;
    return false;
}

__global__ void __launch_bounds__(256) k_mask(MaskArgs a) {
    const int n = a.nc;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    const bool inside = x < n && y < n;
    bool masked = false;
    float c = 0.f;
    size_t v = 0;
    if (inside) {
        v = x + (size_t)n * (y + (size_t)n * z);
        const uint32_t s = __ldcs(a.seeds + v);
        if (s != SEED_EMPTY) {
            const int dx = (int)(s & 0xFF) - x, dy = (int)((s >> 8) & 0xFF) - y, dz = (int)((s >> 16) & 0xFF) - z;
            const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            masked = d2 <= a.T;
        }
        c = __ldcs(a.coarse + v);
    }
    // warp-aggregated append of masked voxels
    const unsigned lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, masked);
    if (bal) {
        uint32_t base = 0;
        const int leader = __ffs(bal) - 1;
        if ((int)lane == leader) base = atomicAdd(a.count, (uint32_t)__popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (masked) a.list[base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)v;
    }
    if (!inside) return;
    const int nf = 2 * n;
    const int n_moved = a.reset ? *a.n_moved : 0;
#pragma unroll
    for (int dz = 0; dz < 2; dz++) {
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const size_t j = (size_t)2 * x + (size_t)nf * ((size_t)(2 * y + dy) + (size_t)nf * (2 * z + dz));
            // the fine grids stream through (each texel once per frame):
            // cache-streaming accesses leave L2 to the tracer's BVH
            float2 u = __ldcs(reinterpret_cast<const float2*>(a.accum + j));
            if (!masked) {
                __stcs(reinterpret_cast<float2*>(a.fine + j), make_float2(c, c));
                if (u.x != CUDART_INF_F || u.y != CUDART_INF_F) {
                    __stcs(reinterpret_cast<float2*>(a.accum + j), make_float2(CUDART_INF_F, CUDART_INF_F));
                    __stcs(reinterpret_cast<uint2*>(a.counts + j), make_uint2(0u, 0u));
                }
                continue;
            }
            float un[2] = {u.x, u.y};
            bool clear[2] = {false, false};
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                if (n_moved > 0 && un[dx] != CUDART_INF_F) {
                    const float px = __fadd_rn(a.bx, __fmul_rn(__fadd_rn((float)(2 * x + dx), 0.5f), a.hf));
                    const float py = __fadd_rn(a.by, __fmul_rn(__fadd_rn((float)(2 * y + dy), 0.5f), a.hf));
                    const float pz = __fadd_rn(a.bz, __fmul_rn(__fadd_rn((float)(2 * z + dz), 0.5f), a.hf));
                    if (near_moved_box(a, x, y, z, px, py, pz, un[dx], n_moved)) {
                        un[dx] = CUDART_INF_F;
                        clear[dx] = true;
                    }
                }
                if (a.alpha != 1.f) {
                    if (a.alpha == 0.f) un[dx] = c;
                    else if (un[dx] != CUDART_INF_F)
                        un[dx] = __fadd_rn(__fmul_rn(a.alpha, un[dx]), __fmul_rn(1.f - a.alpha, c));
                }
            }
            if (un[0] != u.x || un[1] != u.y) __stcs(reinterpret_cast<float2*>(a.accum + j), make_float2(un[0], un[1]));
            if (clear[0] || clear[1]) {
                uint2 cn = __ldcs(reinterpret_cast<const uint2*>(a.counts + j));
                if (clear[0]) cn.x = 0u;
                if (clear[1]) cn.y = 0u;
                __stcs(reinterpret_cast<uint2*>(a.counts + j), cn);
            }
        }
    }
}

}  // namespace

cudaError_t launch_mask(rtsdf_ctx* c, float d_vox) {
    const int n = c->nc;
    cudaError_t e = cudaMemsetAsync(c->d_masked_count, 0, sizeof(uint32_t), c->stream);
    if (e != cudaSuccess) return e;
    MaskArgs a;
    a.seeds = c->seeds[c->cur];
    a.coarse = c->coarse;
    a.nc = n;
    a.T = (long long)mask_threshold(d_vox, c->cfg.beta_vox);
    a.accum = c->accum;
    a.counts = c->counts;
    a.fine = c->fine;
    a.list = c->masked;
    a.count = c->d_masked_count;
    a.alpha = c->cfg.alpha;
    a.boxes = c->obj_box;
    a.moved = c->moved_list;
    a.n_moved = c->d_moved_count;
    a.reset = c->reset_pending && c->n_obj > 0;
    a.bx = c->cfg.bmin[0];
    a.by = c->cfg.bmin[1];
    a.bz = c->cfg.bmin[2];
    a.hf = c->hf;
    a.bin_g = (n + BIN_VOX - 1) / BIN_VOX;
    a.reach = BIN_REACH * c->hc;
    a.bin_start = c->bin_start;
    a.bin_items = c->bin_items;
    a.bin_overflow = c->bin_overflow;
    if (a.reset) {
        BinArgs b;
        b.boxes = c->obj_box;
        b.moved = c->moved_list;
        b.n_moved = c->d_moved_count;
        b.g = a.bin_g;
        b.bx = c->cfg.bmin[0];
        b.by = c->cfg.bmin[1];
        b.bz = c->cfg.bmin[2];
        b.inv_cell = 1.f / (BIN_VOX * c->hc);
        b.reach = a.reach;
        b.count = c->bin_count;
        b.start = c->bin_start;
        b.cursor = c->bin_cursor;
        b.items = c->bin_items;
        b.cap = c->bin_cap;
        b.overflow = c->bin_overflow;
        const size_t cells = (size_t)b.g * b.g * b.g;
        if ((e = cudaMemsetAsync(c->bin_count, 0, cells * sizeof(uint32_t), c->stream))) return e;
        if ((e = cudaMemsetAsync(c->bin_overflow, 0, sizeof(uint32_t), c->stream))) return e;
        const unsigned gb = (unsigned)((c->n_obj + 3) / 4);   // a warp per object, 4 per block
        RTSDF_LAUNCH(c, k_bin_count, gb, 128, 0, b);
        RTSDF_LAUNCH(c, k_bin_scan, 1, 1024, 0, b);
        RTSDF_LAUNCH(c, k_bin_fill, gb, 128, 0, b);
    }
    dim3 block(32, 8, 1), grid((n + 31) / 32, (n + 7) / 8, n);
    RTSDF_LAUNCH(c, k_mask, grid, block, 0, a);
    c->reset_pending = false;
    return cudaGetLastError();
}

}  // namespace rtsdf
