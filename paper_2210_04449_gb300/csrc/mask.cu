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

__device__ __forceinline__ bool near_moved_box(float px, float py, float pz, float u,
                                               const float* __restrict__ boxes,
                                               const int32_t* __restrict__ moved, int n_moved) {
    // fp32, fixed order: d = max(max(lo - p, p - hi), 0); d2 = (dx dx + dy dy) + dz dz
    const float uu = __fmul_rn(u, u);
    for (int i = 0; i < n_moved; i++) {
        const float* b = boxes + 6 * moved[i];
        float dx = fmaxf(fmaxf(__fsub_rn(b[0], px), __fsub_rn(px, b[3])), 0.f);
        float dy = fmaxf(fmaxf(__fsub_rn(b[1], py), __fsub_rn(py, b[4])), 0.f);
        float dz = fmaxf(fmaxf(__fsub_rn(b[2], pz), __fsub_rn(pz, b[5])), 0.f);
        float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (d2 <= uu) return true;
    }
    return false;
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
};

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
        const uint32_t s = a.seeds[v];
        if (s != SEED_EMPTY) {
            const int dx = (int)(s & 0xFF) - x, dy = (int)((s >> 8) & 0xFF) - y, dz = (int)((s >> 16) & 0xFF) - z;
            const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            masked = d2 <= a.T;
        }
        c = a.coarse[v];
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
            float2 u = *reinterpret_cast<const float2*>(a.accum + j);
            if (!masked) {
                *reinterpret_cast<float2*>(a.fine + j) = make_float2(c, c);
                if (u.x != CUDART_INF_F || u.y != CUDART_INF_F) {
                    *reinterpret_cast<float2*>(a.accum + j) = make_float2(CUDART_INF_F, CUDART_INF_F);
                    *reinterpret_cast<uint2*>(a.counts + j) = make_uint2(0u, 0u);
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
                    if (near_moved_box(px, py, pz, un[dx], a.boxes, a.moved, n_moved)) {
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
            if (un[0] != u.x || un[1] != u.y) *reinterpret_cast<float2*>(a.accum + j) = make_float2(un[0], un[1]);
            if (clear[0] || clear[1]) {
                uint2 cn = *reinterpret_cast<const uint2*>(a.counts + j);
                if (clear[0]) cn.x = 0u;
                if (clear[1]) cn.y = 0u;
                *reinterpret_cast<uint2*>(a.counts + j) = cn;
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
    dim3 block(32, 8, 1), grid((n + 31) / 32, (n + 7) / 8, n);
    RTSDF_LAUNCH(c, k_mask, grid, block, 0, a);
    c->reset_pending = false;
    return cudaGetLastError();
}

}  // namespace rtsdf
