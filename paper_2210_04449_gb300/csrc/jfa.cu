// Sec. 2.1 -- 3D jump flooding of the voxel seeds, and the coarse SDF.
//
// Pass with step k: every voxel v reads the previous pass's nearest seed at
// the 27 voxels v + {-k, 0, k}^3 inside the grid and keeps the one with the
// smallest squared distance D2 to v, ties to the smaller packed value
// (= smaller linear index).  Steps are 2^(ceil(log2 N) - 1), ..., 2, 1.
// The last pass also writes the coarse SDF c = h_c sqrt(D2) - beta h_c.
//
// Seeds are packed bytes (x, y, z, 0), so D2 needs two byte dot products:
//   D2 = s.s - 2 s.v + v.v   (dp4a; wraps correctly modulo 2^32, D2 < 2^18)
// and "no seed" (all ones) is pushed above every real distance by OR-ing
// the seed's top byte into D2.  The candidate key is then the pair
// (D2, seed), compared lexicographically.
#include <math_constants.h>

#include "internal.cuh"

namespace rtsdf {
namespace {

__device__ __forceinline__ uint32_t seed_d2(uint32_t s, uint32_t v, uint32_t vv) {
    uint32_t ss = __dp4a(s, s, vv);
    uint32_t sv = __dp4a(s, v, 0u);
    return (ss - 2u * sv) | (s & 0xFF000000u);
}

// Coarse SDF from a packed seed: fp32, h * sqrt(D2) - beta * h, no contraction.
__device__ __forceinline__ float coarse_value(uint32_t best, uint32_t d2, float hc, float beta_h) {
    if (best == SEED_EMPTY) return CUDART_INF_F;
    return __fsub_rn(__fmul_rn(hc, __fsqrt_rn((float)d2)), beta_h);
}

// Tiles of 32 x 8 voxels (x, y) per block, one z-plane per grid z.
template <bool FINAL>
__global__ void __launch_bounds__(256) k_jfa_pass(const uint32_t* __restrict__ in,
                                                 uint32_t* __restrict__ out, int n, int k,
                                                 float* __restrict__ coarse, float hc, float beta_h) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= n || y >= n) return;
    const uint32_t v = pack_seed(x, y, z);
    const uint32_t vv = __dp4a(v, v, 0u);
    uint32_t best = SEED_EMPTY, bestd = 0xFFFFFFFFu;
#pragma unroll
    for (int iz = -1; iz <= 1; iz++) {
        const int zz = z + iz * k;
        if (zz < 0 || zz >= n) continue;
#pragma unroll
        for (int iy = -1; iy <= 1; iy++) {
            const int yy = y + iy * k;
            if (yy < 0 || yy >= n) continue;
            const uint32_t* row = in + (size_t)n * (yy + (size_t)n * zz);
#pragma unroll
            for (int ix = -1; ix <= 1; ix++) {
                const int xx = x + ix * k;
                if (xx < 0 || xx >= n) continue;
                const uint32_t s = __ldg(row + xx);
                const uint32_t d = seed_d2(s, v, vv);
                if (d < bestd || (d == bestd && s < best)) {
                    bestd = d;
                    best = s;
                }
            }
        }
    }
    const size_t idx = x + (size_t)n * (y + (size_t)n * z);
    out[idx] = best;
    if (FINAL) coarse[idx] = coarse_value(best, bestd, hc, beta_h);
}

// Coarse SDF without a pass (N = 1: no jump steps).
__global__ void k_coarse_only(const uint32_t* __restrict__ seeds, size_t n3, int n, float* __restrict__ coarse,
                              float hc, float beta_h) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const uint32_t x = i % n, y = (i / n) % n, z = i / ((size_t)n * n);
    const uint32_t v = pack_seed(x, y, z);
    const uint32_t s = seeds[i];
    coarse[i] = coarse_value(s, seed_d2(s, v, __dp4a(v, v, 0u)), hc, beta_h);
}

}  // namespace

cudaError_t launch_jfa(rtsdf_ctx* c) {
    const int n = c->nc;
    int L = 0;
    while ((1 << L) < n) L++;
    const float beta_h = c->cfg.beta_vox * c->hc;
    dim3 block(32, 8, 1), grid((n + 31) / 32, (n + 7) / 8, n);
    int passes = 0;
    for (int k = L > 0 ? (1 << (L - 1)) : 0; k >= 1; k >>= 1) {
        const uint32_t* in = c->seeds[c->cur];
        uint32_t* out = c->seeds[c->cur ^ 1];
        if (k == 1)
            RTSDF_LAUNCH(c, k_jfa_pass<true>, grid, block, 0, in, out, n, k, c->coarse, c->hc, beta_h);
        else
            RTSDF_LAUNCH(c, k_jfa_pass<false>, grid, block, 0, in, out, n, k, c->coarse, c->hc, beta_h);
        c->cur ^= 1;
        passes++;
    }
    if (passes == 0)
        RTSDF_LAUNCH(c, k_coarse_only, (unsigned)((c->nc3 + 255) / 256), 256, 0, c->seeds[c->cur], c->nc3, n,
                     c->coarse, c->hc, beta_h);
    c->jfa_passes = passes;
    return cudaGetLastError();
}

}  // namespace rtsdf
