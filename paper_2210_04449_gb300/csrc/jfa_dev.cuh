// Device helpers of the 3D jump flood (Sec. 2.1), shared by the per-scene
// pass kernel (jfa.cu) and the batched persistent kernel.
#pragma once

#include <math_constants.h>

#include "internal.cuh"

namespace rtsdf {
namespace dev {

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

// One voxel of a pass with step k (27 candidates, two-pass exact arg-min).
// An offset that leaves the grid is replaced, on that axis only, by offset 0:
// the voxel read is then another member of the same 27-voxel set, so the
// arg-min over the multiset equals the arg-min over the voxels inside the
// grid (voxels outside hold no seed), and no masking is needed.
// NC: read the input through the read-only path (only when no thread of the
// launch writes it).
template <bool FINAL, bool NC>
__device__ __forceinline__ void jfa_voxel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int n, int k,
                                          int x, int y, int z, float* __restrict__ coarse, float hc, float beta_h) {
    const uint32_t v = pack_seed(x, y, z);
    const uint32_t vv = __dp4a(v, v, 0u);
    int xs[3], ys[3], zs[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int o = (i - 1) * k;
        xs[i] = (x + o >= 0 && x + o < n) ? x + o : x;
        ys[i] = (y + o >= 0 && y + o < n) ? y + o : y;
        zs[i] = (z + o >= 0 && z + o < n) ? z + o : z;
    }
    uint32_t cs[27], cd[27];
#pragma unroll
    for (int iz = 0; iz < 3; iz++) {
#pragma unroll
        for (int iy = 0; iy < 3; iy++) {
            const uint32_t* row = in + (size_t)n * (ys[iy] + (size_t)n * zs[iz]);
#pragma unroll
            for (int ix = 0; ix < 3; ix++) {
                const int c = 9 * iz + 3 * iy + ix;
                const uint32_t sv = NC ? __ldg(row + xs[ix]) : row[xs[ix]];
                cs[c] = sv;
                cd[c] = seed_d2(sv, v, vv);
            }
        }
    }
    // smallest D2 (three-input minima), then the smallest seed at that D2
    uint32_t dmin = __vimin3_u32(cd[0], cd[1], cd[2]);
#pragma unroll
    for (int c = 3; c < 27; c += 2) dmin = __vimin3_u32(dmin, cd[c], cd[c + 1]);
    uint32_t best = SEED_EMPTY;
#pragma unroll
    for (int c = 0; c < 27; c++)
        if (cd[c] == dmin) best = min(best, cs[c]);
    const size_t idx = x + (size_t)n * (y + (size_t)n * z);
    out[idx] = best;
    if (FINAL) coarse[idx] = coarse_value(best, dmin, hc, beta_h);
}

}  // namespace dev
}  // namespace rtsdf
