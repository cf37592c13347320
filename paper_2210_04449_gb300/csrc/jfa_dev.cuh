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

// z-blocked pass: a thread floods T voxels of one z-lattice column,
// (x, y, z_t = rz + k (T g + t)) for t < T (jfa_zblock_column; the
// per-scene kernel uses blocks of 32 x 4 threads in (x, y) and
// blockIdx.z = g k + rz).  The T + 2 candidate z-slices (9 voxels
// each) are read once and shared by the column's voxels.
//
// Per candidate seed s = (sx, sy, sz, 0) of a slice, once:
//   A = (sx - x)^2 + (sy - y)^2 + sz^2            vabsdiff4 + dp4a, whose
//       accumulator adds s's top byte (as 0x7F000000): a seedless candidate
//       (all ones) lands above every real key
// Per voxel z_t and candidate, one instruction:
//   key = A - 2 z_t sz = D2 - z_t^2               dp2a.hi (16-bit -2 z_t times byte 2)
// Keys of one voxel share the z_t^2 offset, so their order is D2's; the
// arg-min is the smallest key (three-input signed minima), then the smallest
// seed among the candidates at that key (one clamped add-min and one
// multiply-add per candidate, then unsigned minima) -- the lexicographic
// (D2, seed) minimum.  An x or y offset that leaves the grid reads the voxel's own
// coordinate on that axis (a duplicate of another candidate); a z-slice
// outside the grid holds no seed.  Slices roll through registers: voxel t
// needs slices t .. t + 2 only.
__device__ __forceinline__ int dp2a_hi_s_u(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp2a.hi.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ int vimin3_s(int a, int b, int c) { return __vimin3_s32(a, b, c); }

// the smallest key a seedless candidate can have: A >= 0x7F000000, minus
// 2 z sz with z, sz <= 255
constexpr int SEEDLESS_KEY_MIN = 0x7F000000 - 2 * 255 * 255;

template <bool FINAL, int T>
__device__ __forceinline__ void jfa_zblock_column(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                  int n, int k, int x, int y, int rz, int g,
                                                  float* __restrict__ coarse, float hc, float beta_h) {
    const uint32_t n2 = (uint32_t)n * (uint32_t)n;
    uint32_t xs[3], ys[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int o = (i - 1) * k;
        xs[i] = (uint32_t)((x + o >= 0 && x + o < n) ? x + o : x);
        ys[i] = (uint32_t)((y + o >= 0 && y + o < n) ? y + o : y) * (uint32_t)n;
    }
    const uint32_t vxy = (uint32_t)x | ((uint32_t)y << 8);
    // slice j (0 .. T + 1) holds z-lattice index T g + j - 1
    uint32_t ss[T + 2][9];
    int aa[T + 2][9];
    auto load_slice = [&](int j) {
        const int z = rz + k * (T * g + j - 1);
        if (z >= 0 && z < n) {
            const uint32_t zo = (uint32_t)z * n2;
#pragma unroll
            for (int iy = 0; iy < 3; iy++)
#pragma unroll
                for (int ix = 0; ix < 3; ix++) {
                    const uint32_t sv = __ldg(in + zo + ys[iy] + xs[ix]);
                    const uint32_t d = __vabsdiffu4(sv, vxy);
                    ss[j][3 * iy + ix] = sv;
                    aa[j][3 * iy + ix] = (int)__dp4a(d, d, sv & 0x7F000000u);
                }
        } else {
#pragma unroll
            for (int c = 0; c < 9; c++) {
                ss[j][c] = SEED_EMPTY;
                aa[j][c] = 0x7F000000;
            }
        }
    };
    load_slice(0);
    load_slice(1);
#pragma unroll
    for (int t = 0; t < T; t++) {
        load_slice(t + 2);
        const int z = rz + k * (T * g + t);
        if (z >= n) break;
        // 16-bit -2 z in the low half, 0 in the high half (byte 3 is 0 or, for
        // a seedless candidate, already pushed out of range through A)
        const uint32_t wz = (uint32_t)(-2 * z) & 0xFFFFu;
        int key[27];
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int c = 0; c < 9; c++) key[9 * j + c] = dp2a_hi_s_u(wz, ss[t + j][c], aa[t + j][c]);
        int kmin = vimin3_s(key[0], key[1], key[2]);
#pragma unroll
        for (int c = 3; c < 27; c += 2) kmin = vimin3_s(kmin, key[c], key[c + 1]);
        // smallest seed among the candidates at kmin: gap = min(key - kmin,
        // 255) is 0 exactly for them, and gap * 2^24 + seed then orders every
        // such candidate (a real seed, < 2^24) before every other one (>= 2^24;
        // a seedless one has gap 255 and wraps to 254 * 2^24 + 0xFFFFFF).
        // When kmin itself is a seedless key, every candidate is seedless.
        uint32_t v[27];
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int c = 0; c < 9; c++) {
                const uint32_t gap = (uint32_t)__viaddmin_s32(key[9 * j + c], -kmin, 255);
                v[9 * j + c] = gap * 0x01000000u + ss[t + j][c];
            }
        uint32_t vmin = __vimin3_u32(v[0], v[1], v[2]);
#pragma unroll
        for (int c = 3; c < 27; c += 2) vmin = __vimin3_u32(vmin, v[c], v[c + 1]);
        const uint32_t best = kmin >= SEEDLESS_KEY_MIN ? SEED_EMPTY : vmin;
        const uint32_t idx = (uint32_t)x + ys[1] + (uint32_t)z * n2;
        out[idx] = best;
        if (FINAL) coarse[idx] = dev::coarse_value(best, (uint32_t)(kmin + z * z), hc, beta_h);
    }
}

}  // namespace dev
}  // namespace rtsdf
