// Sec. 2.3 -- soft shadows by sphere tracing the fine SDF, and the
// reverse-mode derivative of that march.
//
// Forward, per shading point p with normal n and unit light direction L:
//   o = p + 2 eps n, t = 0, res = 1, ph = 1e20
//   for i < steps:
//     q = o + t L; stop when q leaves the scene cube
//     h = S(q) (trilinear, cell-centred texels, clamped to the first/last centre)
//     h < eps: visibility 0 (the march met a surface; eps >= one texel, Sec. 2.3)
//     y = h^2 / (2 ph), dd = sqrt(max(h^2 - y^2, 0))
//     t - y > 0: res = min(res, k dd / (t - y))   (triangulation of the
//                current and previous samples, Aaltonen 2018, as in Sec. 2.3)
//     ph = h; t += min(h, step_max)                (restricted step, Sec. 2.3)
//   visibility = clamp(res, 0, 1)
// The grid is gathered through the read-only path; a 1080p floor image at
// 512^3 reads a few hundred MB of texels from L2/L1, not HBM.
//
// Backward: the march is re-run per point (nothing is stored by the forward
// pass), its (t_i, h_i) kept in per-thread local memory, then the single
// penumbra term that produced the visibility (its arg-min step i*) is
// differentiated and swept back to step 0 through h_j = S(o + t_j L) and
// t_{j+1} = t_j + min(h_j, step_max):
//   dsdf[texel] += hbar_j w_texel(q_j)            (fp32 atomics)
//   qbar_j = hbar_j grad S(q_j),  tbar_j += qbar_j . L,  Lbar += t_j qbar_j
// Lbar is reduced per block and mapped through L = v / |v| to the
// unnormalised light vector.  Points stopped by h < eps, points whose res
// stayed 1 and clamped square roots carry no derivative.
#include <math_constants.h>
#include <string.h>

#include "internal.cuh"
#include "trace_dev.cuh"   // Philox-4x32-10

namespace rtsdf {
namespace {

struct ShadowArgs {
    const float* sdf;
    int n;
    float bx, by, bz, ext, inv_h;
    const float* pos;
    const float* nrm;
    long long npix;
    float Lx, Ly, Lz;
    float k, smax, eps;
    int steps;
    float jitter;              // origin jitter toward the light, world units (0: none)
    uint32_t frame, key0, key1;
};

// Sec. 2.3: the origin moves toward the light by xi x jitter, with xi in
// [0, 1) the top 24 bits of the first word of Philox-4x32-10, counter
// (pixel lo, pixel hi, frame, 0x53484457 "SHDW"), key = the context seed.
__device__ __forceinline__ float jitter_shift(const ShadowArgs& a, long long i) {
    uint32_t c[4] = {(uint32_t)i, (uint32_t)((unsigned long long)i >> 32), a.frame, 0x53484457u};
    dev::philox4x32_10(c, a.key0, a.key1);
    return __fmul_rn(__fmul_rn(__uint2float_rn(c[0] >> 8), 0x1p-24f), a.jitter);
}

struct Taps {
    int idx[8];
    float w[8];
    float grad[3];   // d S / d q
};

template <bool GRAD>
__device__ __forceinline__ float sample(const ShadowArgs& a, float qx, float qy, float qz, Taps* tp) {
    const int n = a.n;
    const float q[3] = {qx, qy, qz};
    const float b[3] = {a.bx, a.by, a.bz};
    int i0[3], i1[3];
    float fr[3], dg[3];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        float g = __fsub_rn(__fmul_rn(__fsub_rn(q[ax], b[ax]), a.inv_h), 0.5f);
        dg[ax] = a.inv_h;
        if (!(g > 0.f)) { g = 0.f; dg[ax] = 0.f; }
        if (g >= (float)(n - 1)) { g = (float)(n - 1); dg[ax] = 0.f; }
        int base = (int)floorf(g);
        base = min(base, n - 2);
        base = max(base, 0);
        i0[ax] = base;
        i1[ax] = n > 1 ? base + 1 : 0;
        fr[ax] = n > 1 ? g - (float)base : 0.f;
    }
    float val = 0.f;
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const int x = dx ? i1[0] : i0[0], y = dy ? i1[1] : i0[1], z = dz ? i1[2] : i0[2];
        const float wx = dx ? fr[0] : 1.f - fr[0], wy = dy ? fr[1] : 1.f - fr[1], wz = dz ? fr[2] : 1.f - fr[2];
        const int id = x + n * (y + n * z);
        const float fv = __ldg(a.sdf + id);
        const float w = wx * wy * wz;
        val = fmaf(w, fv, val);
        if (GRAD) {
            tp->idx[c] = id;
            tp->w[c] = w;
            gx = fmaf((dx ? 1.f : -1.f) * wy * wz, fv, gx);
            gy = fmaf(wx * (dy ? 1.f : -1.f) * wz, fv, gy);
            gz = fmaf(wx * wy * (dz ? 1.f : -1.f), fv, gz);
        }
    }
    if (GRAD) {
        tp->grad[0] = gx * dg[0];
        tp->grad[1] = gy * dg[1];
        tp->grad[2] = gz * dg[2];
    }
    return val;
}

__device__ __forceinline__ bool inside(const ShadowArgs& a, float x, float y, float z) {
    return x >= a.bx && x <= a.bx + a.ext && y >= a.by && y <= a.by + a.ext && z >= a.bz && z <= a.bz + a.ext;
}

__global__ void __launch_bounds__(256) k_shadow(ShadowArgs a, float* __restrict__ vis) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= a.npix) return;
    const float two_eps = 2.f * a.eps;
    float ox = fmaf(a.nrm[3 * i], two_eps, a.pos[3 * i]);
    float oy = fmaf(a.nrm[3 * i + 1], two_eps, a.pos[3 * i + 1]);
    float oz = fmaf(a.nrm[3 * i + 2], two_eps, a.pos[3 * i + 2]);
    if (a.jitter != 0.f) {
        const float sh = jitter_shift(a, i);
        ox = fmaf(sh, a.Lx, ox);
        oy = fmaf(sh, a.Ly, oy);
        oz = fmaf(sh, a.Lz, oz);
    }
    float t = 0.f, res = 1.f, ph = 1e20f;
    for (int s = 0; s < a.steps; s++) {
        const float qx = fmaf(t, a.Lx, ox), qy = fmaf(t, a.Ly, oy), qz = fmaf(t, a.Lz, oz);
        if (!inside(a, qx, qy, qz)) break;
        const float h = sample<false>(a, qx, qy, qz, nullptr);
        if (h < a.eps) {
            res = 0.f;
            break;
        }
        const float y = h * h / (2.f * ph);
        const float dd = sqrtf(fmaxf(h * h - y * y, 0.f));
        if (t - y > 0.f) res = fminf(res, a.k * dd / (t - y));
        ph = h;
        t += fminf(h, a.smax);
    }
    vis[i] = fminf(fmaxf(res, 0.f), 1.f);
}

__global__ void __launch_bounds__(128) k_shadow_bwd(ShadowArgs a, const float* __restrict__ dvis,
                                                   float* __restrict__ dsdf, float* __restrict__ dlight,
                                                   float inv_norm) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float lbx = 0.f, lby = 0.f, lbz = 0.f;
    if (i < a.npix && dvis[i] != 0.f) {
        float ts[MAX_SHADOW_STEPS], hs[MAX_SHADOW_STEPS];
        const float two_eps = 2.f * a.eps;
        const float ox = fmaf(a.nrm[3 * i], two_eps, a.pos[3 * i]);
        const float oy = fmaf(a.nrm[3 * i + 1], two_eps, a.pos[3 * i + 1]);
        const float oz = fmaf(a.nrm[3 * i + 2], two_eps, a.pos[3 * i + 2]);
        float t = 0.f, res = 1.f, ph = 1e20f;
        int am = -1;
        bool term = false;
        for (int s = 0; s < a.steps; s++) {
            const float qx = fmaf(t, a.Lx, ox), qy = fmaf(t, a.Ly, oy), qz = fmaf(t, a.Lz, oz);
            if (!inside(a, qx, qy, qz)) break;
            const float h = sample<false>(a, qx, qy, qz, nullptr);
            ts[s] = t;
            hs[s] = h;
            if (h < a.eps) {
                term = true;
                break;
            }
            const float y = h * h / (2.f * ph);
            const float dd = sqrtf(fmaxf(h * h - y * y, 0.f));
            if (t - y > 0.f) {
                const float g = a.k * dd / (t - y);
                if (g < res) {
                    res = g;
                    am = s;
                }
            }
            ph = h;
            t += fminf(h, a.smax);
        }
        if (!term && am >= 0) {
            const int s = am;
            const float h = hs[s], tt = ts[s];
            const float p = s > 0 ? hs[s - 1] : 1e20f;
            const float y = h * h / (2.f * p);
            const float a2 = h * h - y * y;
            if (a2 > 0.f) {
                const float dd = sqrtf(a2), den = tt - y;
                const float dy_dh = h / p, dy_dp = -y / p;
                const float ddd_dh = (h - y * dy_dh) / dd, ddd_dp = (-y * dy_dp) / dd;
                const float gb = dvis[i];
                const float kd = a.k / den, kd2 = a.k * dd / (den * den);
                float hbar = gb * (kd * ddd_dh + kd2 * dy_dh);
                const float pbar = s > 0 ? gb * (kd * ddd_dp + kd2 * dy_dp) : 0.f;
                float tbar = -gb * kd2;
                for (int j = s; j >= 0; j--) {
                    const float tj = ts[j];
                    Taps tp;
                    sample<true>(a, fmaf(tj, a.Lx, ox), fmaf(tj, a.Ly, oy), fmaf(tj, a.Lz, oz), &tp);
#pragma unroll
                    for (int c = 0; c < 8; c++) atomicAdd(dsdf + tp.idx[c], hbar * tp.w[c]);
                    const float qbx = hbar * tp.grad[0], qby = hbar * tp.grad[1], qbz = hbar * tp.grad[2];
                    tbar += qbx * a.Lx + qby * a.Ly + qbz * a.Lz;
                    lbx = fmaf(qbx, tj, lbx);
                    lby = fmaf(qby, tj, lby);
                    lbz = fmaf(qbz, tj, lbz);
                    if (j == 0) break;
                    hbar = (j - 1 == s - 1) ? pbar : 0.f;
                    if (hs[j - 1] < a.smax) hbar += tbar;
                }
            }
        }
    }
    // block reduction of dLoss/dL, then the map through L = v / |v|
    __shared__ float red[3][4];
    for (int off = 16; off >= 1; off >>= 1) {
        lbx += __shfl_xor_sync(0xFFFFFFFFu, lbx, off);
        lby += __shfl_xor_sync(0xFFFFFFFFu, lby, off);
        lbz += __shfl_xor_sync(0xFFFFFFFFu, lbz, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = lbx;
        red[1][w] = lby;
        red[2][w] = lbz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            sx += red[0][k];
            sy += red[1][k];
            sz += red[2][k];
        }
        if (sx != 0.f || sy != 0.f || sz != 0.f) {
            const float dl = sx * a.Lx + sy * a.Ly + sz * a.Lz;
            atomicAdd(dlight + 0, (sx - dl * a.Lx) * inv_norm);
            atomicAdd(dlight + 1, (sy - dl * a.Ly) * inv_norm);
            atomicAdd(dlight + 2, (sz - dl * a.Lz) * inv_norm);
        }
    }
}

// Temporal anti-aliasing of a visibility image (Sec. 2.3 steadies the
// jitter noise with TAA), static camera: the history is clamped to the
// current frame's 3x3 neighbourhood range (clamped at the border) and
// blended toward the current value in place, h = hc + blend (cur - hc).
__global__ void __launch_bounds__(256) k_taa(const float* __restrict__ cur, float* __restrict__ hist, int w,
                                             int h, float blend) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    if (x >= w || y >= h) return;
    float mn = CUDART_INF_F, mx = -CUDART_INF_F;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
        const int yy = min(max(y + dy, 0), h - 1);
#pragma unroll
        for (int dx = -1; dx <= 1; dx++) {
            const int xx = min(max(x + dx, 0), w - 1);
            const float v = __ldg(cur + (size_t)yy * w + xx);
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
    }
    const size_t i = (size_t)y * w + x;
    const float c = __ldg(cur + i);
    const float hc = fminf(fmaxf(hist[i], mn), mx);
    hist[i] = fmaf(blend, __fsub_rn(c, hc), hc);
}

ShadowArgs make_args(rtsdf_ctx* c, const float* sdf, const float* pos, const float* nrm, int64_t npix,
                     const float L[3], float k, int steps, float smax, float eps) {
    ShadowArgs a;
    a.sdf = sdf ? sdf : c->fine;
    a.n = c->nf;
    a.bx = c->cfg.bmin[0];
    a.by = c->cfg.bmin[1];
    a.bz = c->cfg.bmin[2];
    a.ext = c->cfg.extent;
    a.inv_h = (float)c->nf / c->cfg.extent;
    a.pos = pos;
    a.nrm = nrm;
    a.npix = npix;
    a.Lx = L[0];
    a.Ly = L[1];
    a.Lz = L[2];
    a.k = k;
    a.smax = smax;
    a.eps = eps;
    a.steps = steps;
    a.jitter = 0.f;
    a.frame = 0;
    a.key0 = (uint32_t)c->cfg.seed;
    a.key1 = (uint32_t)(c->cfg.seed >> 32);
    return a;
}

// Thin-surface fallback (Sec. 3: the march can step through a surface
// thinner than its epsilon and leave a hole in the umbra; the paper would
// shadow-map such regions).  Exact occlusion of the ray from the march's
// origin fmaf(n, 2 eps, p) along L: a BVH traversal that stops at the first
// hit (any hit decides), with the tracer's box and ray/triangle tests.  A
// blocked point gets visibility 0; the others keep the march's value.
// TEX: node fetches split between the load and texture pipes, as in the
// tracer.
template <bool TEX>
__global__ void __launch_bounds__(dev::TRACE_THREADS) k_shadow_exact(dev::TraceArgs t, const float* __restrict__ pos,
                                                                     const float* __restrict__ nrm, long long npix,
                                                                     float Lx, float Ly, float Lz, float two_eps,
                                                                     float* vis, uint8_t* blocked) {
    __shared__ int2 s_stack[dev::SMEM_STACK][dev::TRACE_THREADS];
    int2 deep[TRACE_STACK - dev::SMEM_STACK];
    dev::Stack stk{&s_stack[0][threadIdx.x], deep};
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npix) return;                      // no barrier below
    dev::Ray r;
    r.o = make_float3(fmaf(nrm[3 * i], two_eps, pos[3 * i]), fmaf(nrm[3 * i + 1], two_eps, pos[3 * i + 1]),
                      fmaf(nrm[3 * i + 2], two_eps, pos[3 * i + 2]));
    r.d = make_float3(Lx, Ly, Lz);
    r.id = make_float3(dev::safe_inv(Lx), dev::safe_inv(Ly), dev::safe_inv(Lz));
    r.oid = make_float3(r.o.x * r.id.x, r.o.y * r.id.y, r.o.z * r.id.z);
    r.bt = CUDART_INF_F;
    r.bidx = 0x7FFFFFFF;
    r.bfront = false;
    r.node = t.nt > 1 ? 0 : WIDE_EMPTY;
    r.leaf = t.nt == 1 ? 0 : WIDE_EMPTY;
    r.sp = 0;
    r.slot = 0;
    r.steps = 0;
    uint32_t nv = 0, ntest = 0;
    // every step enters a node or tests a leaf (bounded by the step guard);
    // the loop ends at the first hit or when nothing is left
    while (r.bidx == 0x7FFFFFFF && !dev::ray_done(r)) {
        dev::node_step<false, TEX>(t, r, stk, nv);
        if (r.leaf != WIDE_EMPTY) dev::leaf_step<false>(t, r, stk, nv, ntest);
        dev::step_guard(t, r);
    }
    const bool b = r.bidx != 0x7FFFFFFF;
    if (blocked) blocked[i] = (uint8_t)b;
    if (b && vis) vis[i] = 0.f;
}

}  // namespace

cudaError_t launch_shadow(rtsdf_ctx* c, const float* sdf, const float* pos, const float* nrm, int64_t npix,
                          const float L[3], float k, int steps, float smax, float eps, float jitter, int frame,
                          float* vis) {
    if (npix == 0) return cudaSuccess;
    ShadowArgs a = make_args(c, sdf, pos, nrm, npix, L, k, steps, smax, eps);
    a.jitter = jitter;
    a.frame = (uint32_t)frame;
    RTSDF_LAUNCH(c, k_shadow, (unsigned)((npix + 255) / 256), 256, 0, a, vis);
    return cudaGetLastError();
}

cudaError_t launch_shadow_bwd(rtsdf_ctx* c, const float* sdf, const float* pos, const float* nrm, int64_t npix,
                              const float L[3], float inv_norm, float k, int steps, float smax, float eps,
                              const float* dvis, float* dsdf, float* dlight) {
    if (npix == 0) return cudaSuccess;
    ShadowArgs a = make_args(c, sdf, pos, nrm, npix, L, k, steps, smax, eps);
    RTSDF_LAUNCH(c, k_shadow_bwd, (unsigned)((npix + 127) / 128), 128, 0, a, dvis, dsdf, dlight, inv_norm);
    return cudaGetLastError();
}

cudaError_t launch_taa(rtsdf_ctx* c, const float* cur, float* hist, int w, int h, float blend) {
    if (w == 0 || h == 0) return cudaSuccess;
    dim3 block(32, 8, 1), grid((unsigned)((w + 31) / 32), (unsigned)((h + 7) / 8), 1);
    RTSDF_LAUNCH(c, k_taa, grid, block, 0, cur, hist, w, h, blend);
    return cudaGetLastError();
}

cudaError_t launch_shadow_exact(rtsdf_ctx* c, const float* pos, const float* nrm, int64_t npix, const float L[3],
                                float eps, float* vis, uint8_t* blocked) {
    if (npix == 0) return cudaSuccess;
    dev::TraceArgs t;
    memset(&t, 0, sizeof(t));
    t.wide = c->bvh.wide;
    t.wtex = texture_fetch_on() ? c->bvh.wtex : 0;
    t.tri = c->bvh.tri;
    t.nt = c->bvh.nt;
    t.err = c->d_err;
    const unsigned g = (unsigned)((npix + dev::TRACE_THREADS - 1) / dev::TRACE_THREADS);
    if (t.wtex)
        RTSDF_LAUNCH(c, k_shadow_exact<true>, g, dev::TRACE_THREADS, 0, t, pos, nrm, (long long)npix, L[0], L[1],
                     L[2], 2.f * eps, vis, blocked);
    else
        RTSDF_LAUNCH(c, k_shadow_exact<false>, g, dev::TRACE_THREADS, 0, t, pos, nrm, (long long)npix, L[0], L[1],
                     L[2], 2.f * eps, vis, blocked);
    return cudaGetLastError();
}

}  // namespace rtsdf
