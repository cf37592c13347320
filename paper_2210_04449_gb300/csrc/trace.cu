// Sec. 2.2 -- ray tracing of the masked fine texels with temporal
// accumulation (Eq. 1) and the front/back sign vote.
//
// Work layout: the mask kernel lists masked coarse voxels; each contributes
// its 8 fine children.  A group of G = min(R, 32) lanes of a warp owns one
// texel and its R rays (R / G rays per lane), so 32 / G texels share a warp.
// Each lane
//   * draws its directions from Philox-4x32-10 (Salmon et al., SC'11) with
//     counter (draw, ray, frame, texel) and key (seed lo, seed hi), mapped to
//     the sphere by Marsaglia's (1972) rejection method -- integer accept
//     test, fp32 map, so every direction is bit-reproducible;
//   * finds the closest hit by a stack traversal of the binary BVH (both
//     child boxes per node fetch, nearer child first, the farther one pushed
//     with its entry distance and skipped on pop when it can no longer hold
//     a closer hit), testing leaves with Moller-Trumbore in fp32 with the
//     operation order written out (explicit fma / rounding intrinsics);
//     equal distances keep the smaller original triangle index.
// The group then reduces (min distance, #front, #back) with shuffles and its
// first lane applies u_t = min(u, r_t) (Eq. 1; the alpha decay was applied by
// the mask kernel), adds the counts and writes f_t = +-u_t (c_t while no ray
// has hit), negative when back hits outnumber front hits.
#include <math_constants.h>

#include "internal.cuh"

namespace rtsdf {
namespace {

struct TraceArgs {
    const uint32_t* masked;
    const uint32_t* count;
    int nc;
    int rays, log2_group, rays_per_lane;
    uint32_t key0, key1, frame;
    float bx, by, bz, hf;
    const BNode* nodes;
    const float4* tri;
    long long nt;
    const float* coarse;
    float* accum;
    uint32_t* counts;
    float* fine;
    uint32_t* err;
    TraceCounters* counters;   // work counters (counting variant only)
};

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ bool marsaglia(uint32_t wa, uint32_t wb, float3& d) {
    const int A = 2 * (int)(wa >> 9) + 1 - (1 << 23);
    const int B = 2 * (int)(wb >> 9) + 1 - (1 << 23);
    const long long S = (long long)A * A + (long long)B * B;
    if (S >= (1LL << 46)) return false;
    const float s = __fmul_rn(__ll2float_rn(S), 0x1p-46f);
    const float root = __fsqrt_rn(__fsub_rn(1.0f, s));
    const float a = __fmul_rn(__int2float_rn(A), 0x1p-23f);
    const float b = __fmul_rn(__int2float_rn(B), 0x1p-23f);
    d.x = __fmul_rn(__fmul_rn(2.0f, a), root);
    d.y = __fmul_rn(__fmul_rn(2.0f, b), root);
    d.z = __fsub_rn(1.0f, __fmul_rn(2.0f, s));
    return true;
}

__device__ __forceinline__ float3 sphere_dir(uint32_t k0, uint32_t k1, uint32_t texel, uint32_t frame,
                                             uint32_t ray) {
    float3 d;
    for (uint32_t draw = 0; draw < 8; draw++) {
        uint32_t c[4] = {draw, ray, frame, texel};
        philox4x32_10(c, k0, k1);
        if (marsaglia(c[0], c[1], d)) return d;
        if (marsaglia(c[2], c[3], d)) return d;
    }
    return make_float3(0.f, 0.f, 1.f);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                       __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}

// Moller-Trumbore, closed triangle, t >= 0.  Returns hit; t and front out.
__device__ __forceinline__ bool ray_tri(float3 o, float3 d, float3 v0, float3 e1, float3 e2, float& t,
                                       bool& front) {
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    if (det == 0.0f) return false;
    const float inv = __fdiv_rn(1.0f, det);
    const float3 tv = make_float3(__fsub_rn(o.x, v0.x), __fsub_rn(o.y, v0.y), __fsub_rn(o.z, v0.z));
    const float u = __fmul_rn(dot3(tv, p), inv);
    if (!(u >= 0.0f && u <= 1.0f)) return false;
    const float3 q = cross3(tv, e1);
    const float v = __fmul_rn(dot3(d, q), inv);
    if (!(v >= 0.0f && __fadd_rn(u, v) <= 1.0f)) return false;
    const float tt = __fmul_rn(dot3(e2, q), inv);
    if (!(tt >= 0.0f)) return false;
    t = tt;
    front = det > 0.0f;
    return true;
}

__device__ __forceinline__ float safe_inv(float d) {
    return __fdiv_rn(1.0f, fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d);
}

struct Hit {
    float t;
    int idx;
    bool front;
};

template <bool COUNT>
__device__ __forceinline__ void closest_hit(const TraceArgs& a, float3 o, float3 d, Hit& h, uint32_t& visits_out,
                                            uint32_t& tests_out) {
    h.t = CUDART_INF_F;
    h.idx = 0x7FFFFFFF;
    h.front = false;
    if (a.nt == 0) return;
    const float3 id = make_float3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    const float3 oid = make_float3(o.x * id.x, o.y * id.y, o.z * id.z);
    int2 stack[TRACE_STACK];
    int sp = 0;
    int node = a.nt > 1 ? 0 : ~0;
    // every node is entered at most once per ray (2 nt - 1 nodes); the bound
    // only guards against a damaged tree
    for (long long visits = 0;; visits++) {
        if (visits > 2 * a.nt) {
            atomicOr(a.err, ERR_STACK);
            return;
        }
        if (COUNT) visits_out++;
        if (node >= 0) {
            const float4 na = __ldg(&a.nodes[node].a);
            const float4 nb = __ldg(&a.nodes[node].b);
            const float4 nc = __ldg(&a.nodes[node].c);
            const int4 nd = __ldg(&a.nodes[node].d);
            // left child box: (na.x, na.y) x, (na.z, na.w) y, (nc.x, nc.y) z
            float x0 = fmaf(na.x, id.x, -oid.x), x1 = fmaf(na.y, id.x, -oid.x);
            float y0 = fmaf(na.z, id.y, -oid.y), y1 = fmaf(na.w, id.y, -oid.y);
            float z0 = fmaf(nc.x, id.z, -oid.z), z1 = fmaf(nc.y, id.z, -oid.z);
            const float tl0 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), 0.f));
            const float tl1 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), h.t));
            x0 = fmaf(nb.x, id.x, -oid.x); x1 = fmaf(nb.y, id.x, -oid.x);
            y0 = fmaf(nb.z, id.y, -oid.y); y1 = fmaf(nb.w, id.y, -oid.y);
            z0 = fmaf(nc.z, id.z, -oid.z); z1 = fmaf(nc.w, id.z, -oid.z);
            const float tr0 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), 0.f));
            const float tr1 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), h.t));
            const bool hl = tl0 <= tl1, hr = tr0 <= tr1;
            if (hl && hr) {
                const bool lfirst = tl0 <= tr0;
                const int far = lfirst ? nd.y : nd.x;
                const float tfar = lfirst ? tr0 : tl0;
                if (sp < TRACE_STACK) stack[sp++] = make_int2(far, __float_as_int(tfar));
                else atomicOr(a.err, ERR_STACK);
                node = lfirst ? nd.x : nd.y;
                continue;
            }
            if (hl) { node = nd.x; continue; }
            if (hr) { node = nd.y; continue; }
        } else {
            const int leaf = ~node;
            if (COUNT) tests_out++;
            const float4 p0 = __ldg(&a.tri[3 * leaf]);
            const float4 p1 = __ldg(&a.tri[3 * leaf + 1]);
            const float4 p2 = __ldg(&a.tri[3 * leaf + 2]);
            float t;
            bool fr;
            if (ray_tri(o, d, make_float3(p0.x, p0.y, p0.z), make_float3(p1.x, p1.y, p1.z),
                        make_float3(p2.x, p2.y, p2.z), t, fr)) {
                const int idx = __float_as_int(p0.w);
                if (t < h.t || (t == h.t && idx < h.idx)) {
                    h.t = t;
                    h.idx = idx;
                    h.front = fr;
                }
            }
        }
        // pop the next candidate that can still hold a hit at distance <= h.t
        for (;;) {
            if (sp == 0) return;
            const int2 e = stack[--sp];
            if (__int_as_float(e.y) <= h.t) {
                node = e.x;
                break;
            }
        }
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(128) k_trace(TraceArgs a) {
    uint32_t n_rays = 0, n_visits = 0, n_tests = 0;
    const uint32_t n_vox = *a.count;
    const uint64_t n_tex = (uint64_t)n_vox * 8u;
    const int G = 1 << a.log2_group;              // lanes per texel
    const int tpw = 32 >> a.log2_group;           // texels per warp
    const unsigned lane = threadIdx.x & 31;
    const unsigned sub = lane & (G - 1);
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (gridDim.x * (uint64_t)blockDim.x) >> 5;
    const int nf = 2 * a.nc;
    for (uint64_t base = warp * tpw; base < n_tex; base += nwarps * tpw) {
        const uint64_t slot = base + (lane >> a.log2_group);
        const bool valid = slot < n_tex;
        float rmin = CUDART_INF_F;
        uint32_t nfr = 0, nbk = 0;
        uint32_t texel = 0;
        uint32_t parent = 0;
        if (valid) {
            parent = a.masked[slot >> 3];
            const uint32_t ch = (uint32_t)(slot & 7);
            const uint32_t px = parent % a.nc, py = (parent / a.nc) % a.nc, pz = parent / (a.nc * a.nc);
            const uint32_t jx = 2 * px + (ch & 1), jy = 2 * py + ((ch >> 1) & 1), jz = 2 * pz + (ch >> 2);
            texel = jx + nf * (jy + nf * jz);
            const float3 o = make_float3(__fadd_rn(a.bx, __fmul_rn(__fadd_rn((float)jx, 0.5f), a.hf)),
                                         __fadd_rn(a.by, __fmul_rn(__fadd_rn((float)jy, 0.5f), a.hf)),
                                         __fadd_rn(a.bz, __fmul_rn(__fadd_rn((float)jz, 0.5f), a.hf)));
            for (int k = 0; k < a.rays_per_lane; k++) {
                const uint32_t ray = sub + (uint32_t)k * G;
                const float3 d = sphere_dir(a.key0, a.key1, texel, a.frame, ray);
                Hit h;
                closest_hit<COUNT>(a, o, d, h, n_visits, n_tests);
                if (COUNT) n_rays++;
                if (h.idx != 0x7FFFFFFF) {
                    rmin = fminf(rmin, h.t);
                    if (h.front) nfr++;
                    else nbk++;
                }
            }
        }
        // reduce over the G lanes of the texel group
        for (int off = G >> 1; off >= 1; off >>= 1) {
            rmin = fminf(rmin, __shfl_xor_sync(0xFFFFFFFFu, rmin, off));
            nfr += __shfl_xor_sync(0xFFFFFFFFu, nfr, off);
            nbk += __shfl_xor_sync(0xFFFFFFFFu, nbk, off);
        }
        if (valid && sub == 0) {
            const float u = fminf(a.accum[texel], rmin);
            const uint32_t cw = a.counts[texel];
            const uint32_t f = min((cw & 0xFFFFu) + nfr, 0xFFFFu);
            const uint32_t b = min((cw >> 16) + nbk, 0xFFFFu);
            a.accum[texel] = u;
            a.counts[texel] = f | (b << 16);
            const float mag = u == CUDART_INF_F ? a.coarse[parent] : u;
            a.fine[texel] = b > f ? -mag : mag;
        }
    }
    if (COUNT) {
        unsigned long long r = n_rays, v = n_visits, t = n_tests;
        for (int off = 16; off >= 1; off >>= 1) {
            r += __shfl_xor_sync(0xFFFFFFFFu, r, off);
            v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
            t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&a.counters->rays, r);
            atomicAdd(&a.counters->visits, v);
            atomicAdd(&a.counters->tests, t);
        }
    }
}

}  // namespace

cudaError_t launch_trace(rtsdf_ctx* c, int rays, int frame) {
    TraceArgs a;
    a.masked = c->masked;
    a.count = c->d_masked_count;
    a.nc = c->nc;
    a.rays = rays;
    int lg = 0;
    while ((1 << lg) < rays) lg++;
    a.log2_group = lg < 5 ? lg : 5;
    a.rays_per_lane = rays >> a.log2_group;
    a.key0 = (uint32_t)c->cfg.seed;
    a.key1 = (uint32_t)(c->cfg.seed >> 32);
    a.frame = (uint32_t)frame;
    a.bx = c->cfg.bmin[0];
    a.by = c->cfg.bmin[1];
    a.bz = c->cfg.bmin[2];
    a.hf = c->hf;
    a.nodes = c->bvh.nodes;
    a.tri = c->bvh.tri;
    a.nt = c->bvh.nt;
    a.coarse = c->coarse;
    a.accum = c->accum;
    a.counts = c->counts;
    a.fine = c->fine;
    a.err = c->d_err;
    a.counters = c->d_counters;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const unsigned grid = (unsigned)(sms > 0 ? sms : 132) * 16u;
    if (c->counting) RTSDF_LAUNCH(c, k_trace<true>, grid, 128, 0, a);
    else RTSDF_LAUNCH(c, k_trace<false>, grid, 128, 0, a);
    return cudaGetLastError();
}

}  // namespace rtsdf
