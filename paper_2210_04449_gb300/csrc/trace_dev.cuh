// Device helpers of the Sec. 2.2 tracer (ray generation, ray/triangle test,
// 4-wide BVH traversal step), shared by the per-scene tracer (trace.cu) and
// the batched persistent kernel.
#pragma once

#include <math_constants.h>

#include "internal.cuh"

namespace rtsdf {
namespace dev {

struct TraceArgs {
    const uint32_t* masked;
    const uint32_t* count;
    int nc;
    int rays, log2_rays;
    uint32_t key0, key1, frame;
    float bx, by, bz, hf;
    const WNode* wide;
    cudaTextureObject_t wtex;  // the same nodes as int4 texels (used when the kernel's TEX is set)
    const float4* tri;
    long long nt;
    const float* coarse;
    float* accum;
    uint32_t* counts;
    float* fine;
    uint32_t* err;
    TraceCounters* counters;   // work counters (counting variant only)
    uint32_t* ray_min;         // [8 nc^3] per texel slot: min hit distance bits of this frame
    uint32_t* ray_cnt;         // [8 nc^3] per texel slot: front | back << 16 hits of this frame
    unsigned long long* next_ray;
    int refill_min;            // refill a warp once this many lanes are idle
    int ray_chunk;             // rays a warp takes from the global counter at a time
    int leaf_min;              // run the leaf phase once this many lanes hold a parked leaf
    uint32_t nc_mag;           // ceil(2^32 / nc): umulhi(v, nc_mag) = v / nc for v < 2^24
    int nearest;               // sign from the nearest hit's face; rays capped at the texel's u
};

// Per-slot "nothing committed" value of ray_min: +inf bits for the vote,
// all ones for the nearest-face key (t bits << 1 | back).
__host__ __device__ constexpr uint32_t ray_min_none(bool nearest) { return nearest ? 0xFFFFFFFFu : 0x7F800000u; }

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
    // every quantity is computed (the same operations in the same order as
    // a test with early exits), and the accept conditions are combined at
    // the end: with the lanes of a warp on different triangles, the early
    // exits would only add branches
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    const float inv = __fdiv_rn(1.0f, det);
    const float3 tv = make_float3(__fsub_rn(o.x, v0.x), __fsub_rn(o.y, v0.y), __fsub_rn(o.z, v0.z));
    const float u = __fmul_rn(dot3(tv, p), inv);
    const float3 q = cross3(tv, e1);
    const float v = __fmul_rn(dot3(d, q), inv);
    const float tt = __fmul_rn(dot3(e2, q), inv);
    const bool ok = (det != 0.0f) & (u >= 0.0f) & (u <= 1.0f) & (v >= 0.0f) & (__fadd_rn(u, v) <= 1.0f) &
                    (tt >= 0.0f);
    t = tt;
    front = det > 0.0f;
    return ok;
}

// Reciprocal of a direction component for the box tests only (an
// approximate reciprocal is enough: the same value serves every box of the
// ray and the leaf boxes are padded); zero components become +-1e30.
__device__ __forceinline__ float safe_inv(float d) {
    return __fdividef(1.0f, fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d);
}

// 256-bit read-only global load (sm_100 and later) of two float4 at a
// 32-byte aligned address.
__device__ __forceinline__ void ldg256(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Three-input fp32 maximum / minimum (sm_100 and later); like fmaxf /
// fminf, a NaN operand is ignored.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Per-lane ray state of the persistent tracer.
struct Ray {
    float3 o, d, id, oid;
    float bt;          // closest hit distance so far
    int bidx;          // its original triangle index (0x7FFFFFFF: none)
    bool bfront;
    int node;          // next node to enter (>= 0 internal, < 0 ~leaf, WIDE_EMPTY none)
    int leaf;          // parked leaf waiting for the leaf phase (WIDE_EMPTY none)
    int sp;
    uint32_t slot;     // texel slot = 8 * (masked-list position) + child
    uint32_t steps;    // nodes entered; a tree of 2 nt - 1 nodes bounds it
};

__device__ __forceinline__ void setup_ray(const TraceArgs& a, uint64_t g, Ray& r) {
    const uint32_t slot = (uint32_t)(g >> a.log2_rays);
    const uint32_t ray = (uint32_t)(g & (uint64_t)(a.rays - 1));
    const uint32_t parent = a.masked[slot >> 3];
    const uint32_t ch = slot & 7u;
    const uint32_t nc = (uint32_t)a.nc, nf = 2u * nc;
    const uint32_t pq = __umulhi(parent, a.nc_mag), pz = __umulhi(pq, a.nc_mag);
    const uint32_t px = parent - pq * nc, py = pq - pz * nc;
    const uint32_t jx = 2 * px + (ch & 1), jy = 2 * py + ((ch >> 1) & 1), jz = 2 * pz + (ch >> 2);
    const uint32_t texel = jx + nf * (jy + nf * jz);
    // nearest-face variant: no hit beyond the texel's accumulated distance
    // can change its result, so the ray starts with that distance as its
    // best hit (hits at exactly that distance still count: bidx is unset)
    const float cap = a.nearest ? a.accum[texel] : CUDART_INF_F;
    r.o = make_float3(__fadd_rn(a.bx, __fmul_rn(__fadd_rn((float)jx, 0.5f), a.hf)),
                      __fadd_rn(a.by, __fmul_rn(__fadd_rn((float)jy, 0.5f), a.hf)),
                      __fadd_rn(a.bz, __fmul_rn(__fadd_rn((float)jz, 0.5f), a.hf)));
    r.d = sphere_dir(a.key0, a.key1, texel, a.frame, ray);
    r.id = make_float3(safe_inv(r.d.x), safe_inv(r.d.y), safe_inv(r.d.z));
    r.oid = make_float3(r.o.x * r.id.x, r.o.y * r.id.y, r.o.z * r.id.z);
    r.bt = cap;
    r.bidx = 0x7FFFFFFF;
    r.bfront = false;
    // the root; a one-triangle mesh has no node, so its leaf starts parked
    // (a ray with neither a node nor a parked leaf is done)
    r.node = a.nt > 1 ? 0 : WIDE_EMPTY;
    r.leaf = a.nt == 1 ? 0 : WIDE_EMPTY;
    r.sp = 0;
    r.slot = slot;
    r.steps = 0;
}

constexpr int TRACE_THREADS = 128;
constexpr int SMEM_STACK = 24;

// Traversal stack of one lane: (node, entry distance) pairs, the first
// SMEM_STACK in shared memory laid out [entry][thread] (a push or pop of a
// warp is one 64-bit access per lane over distinct banks), deeper entries
// in local memory.
struct Stack {
    int2* e;      // &s_stack[0][thread], stride TRACE_THREADS
    int2* deep;   // local overflow
    __device__ __forceinline__ void push(int sp, int node, float t0) {
        const int2 v = make_int2(node, __float_as_int(t0));
        if (sp < SMEM_STACK) e[sp * TRACE_THREADS] = v;
        else deep[sp - SMEM_STACK] = v;
    }
    __device__ __forceinline__ void pop(int sp, int& node, float& t0) const {
        const int2 v = sp < SMEM_STACK ? e[sp * TRACE_THREADS] : deep[sp - SMEM_STACK];
        node = v.x;
        t0 = __int_as_float(v.y);
    }
};

// Traversal in two phases.  With one triangle per leaf, a warp in which
// every lane takes either a node step or a leaf step would pay both paths on
// almost every iteration.  So a lane that reaches a leaf parks it (one per
// lane) and keeps entering internal nodes; the warp runs the leaf phase only
// when enough lanes hold a parked leaf or some cannot continue.  The order of
// triangle tests does not change the closest hit (every triangle whose box
// the ray meets is tested unless its entry distance exceeds the best hit).

// Pop the next entry that can still hold a hit at distance <= bt, parking
// leaves while the lane's slot is free; stops at an internal node, at a leaf
// behind the parked one, or with the stack empty (r.node = WIDE_EMPTY).
__device__ __forceinline__ void advance(Ray& r, Stack& stack) {
    int nx = WIDE_EMPTY;
    while (r.sp > 0) {
        int cand;
        float te;
        stack.pop(--r.sp, cand, te);
        if (te > r.bt) continue;
        if (cand < 0 && r.leaf == WIDE_EMPTY) {
            r.leaf = ~cand;
            continue;
        }
        nx = cand;
        break;
    }
    r.node = nx;
}

__device__ __forceinline__ bool ray_done(const Ray& r) { return r.node == WIDE_EMPTY && r.leaf == WIDE_EMPTY; }

// A damaged tree (a cycle) would make a walk endless: a lane whose walk has
// taken more node and leaf steps than a tree of 2 nt - 1 nodes allows stops,
// and the call reports ERR_STACK.  Checked once per traversal iteration.
template <class A>
__device__ __forceinline__ void step_guard(const A& a, Ray& r) {
    if (r.steps > 2u * (uint32_t)a.nt + 2u) {
        atomicOr(a.err, ERR_STACK);
        r.node = r.leaf = WIDE_EMPTY;
    }
}

// Enter r.node if it is an internal node (A: any argument block with the BVH
// fields wide, wtex, tri, nt and err).  TEX: the child ids come through the
// texture pipe (wtex), the box planes through the load pipe.
template <bool COUNT, bool TEX, class A>
__device__ __forceinline__ void node_step(const A& a, Ray& r, Stack& stack, uint32_t& visits) {
    const int node = r.node;
    if (node < 0) return;   // none, or a leaf waiting behind the parked one
    r.steps++;
    if (COUNT) visits++;
    // 4-wide node: test the four child boxes, visit the nearest hit child
    // next and push the others farthest-first with their entry distance.
    // Near / far plane rows are chosen by the ray's direction signs (rows:
    // lox, hix, loy, hiy, loz, hiz), so each slab needs no min/max of its two
    // planes; an empty slot (lo = +inf, hi = -inf) never hits.
    // Each axis's (lo, hi) row pair is one aligned 32-byte sector fetched by
    // a single 256-bit load: with the lanes of a warp on different nodes, the
    // L1's load/store data pipe spends one wavefront per lane and sector, not
    // per 16 bytes, and that pipe binds the traversal.  The texture pipe has
    // its own: with TEX, the child ids (the node's fourth sector) are fetched
    // as an int4 texel through it, 3.7 % faster on the 1M-triangle frame.
    const WNode* w = a.wide + node;
    const float4* row = &w->lox;
    float4 lx, hx, ly, hy, lz, hz;
    ldg256(row, lx, hx);
    ldg256(row + 2, ly, hy);
    ldg256(row + 4, lz, hz);
    int4 ch;
    if constexpr (TEX) ch = tex1Dfetch<int4>(a.wtex, 8 * node + 6);
    else ch = __ldg(&w->child);
    const bool sx = r.id.x < 0.f, sy = r.id.y < 0.f, sz = r.id.z < 0.f;
    const float4 nx = sx ? hx : lx, fx = sx ? lx : hx;
    const float4 ny = sy ? hy : ly, fy = sy ? ly : hy;
    const float4 nz = sz ? hz : lz, fz = sz ? lz : hz;
    float key[4];
    int val[4] = {ch.x, ch.y, ch.z, ch.w};
    const float bnx[4] = {nx.x, nx.y, nx.z, nx.w}, bfx[4] = {fx.x, fx.y, fx.z, fx.w};
    const float bny[4] = {ny.x, ny.y, ny.z, ny.w}, bfy[4] = {fy.x, fy.y, fy.z, fy.w};
    const float bnz[4] = {nz.x, nz.y, nz.z, nz.w}, bfz[4] = {fz.x, fz.y, fz.z, fz.w};
    int nh = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float t0 = fmax3(fmaf(bnx[k], r.id.x, -r.oid.x), fmaf(bny[k], r.id.y, -r.oid.y),
                               fmaxf(fmaf(bnz[k], r.id.z, -r.oid.z), 0.f));
        const float t1 = fmin3(fmaf(bfx[k], r.id.x, -r.oid.x), fmaf(bfy[k], r.id.y, -r.oid.y),
                               fminf(fmaf(bfz[k], r.id.z, -r.oid.z), r.bt));
        const bool hit = t0 <= t1;
        key[k] = hit ? t0 : CUDART_INF_F;
        nh += hit;
    }
    // ascending sort of (key, val) by a 5-exchange network, done whether or
    // not a child was hit (a branch around it costs more than it saves)
#define RTSDF_CAS(i, j)                                                     \
    if (key[j] < key[i]) {                                                  \
        const float tk = key[i]; key[i] = key[j]; key[j] = tk;              \
        const int tv = val[i]; val[i] = val[j]; val[j] = tv;                \
    }
    RTSDF_CAS(0, 1) RTSDF_CAS(2, 3) RTSDF_CAS(0, 2) RTSDF_CAS(1, 3) RTSDF_CAS(1, 2)
#undef RTSDF_CAS
    // a nearest child that is a leaf is parked at once when the lane's slot
    // is free, and the next nearest is entered without a round trip through
    // the stack
    const int first = (nh > 0 && val[0] < 0 && r.leaf == WIDE_EMPTY) ? 1 : 0;
    if (first) r.leaf = ~val[0];
#pragma unroll
    for (int k = 3; k >= 1; k--) {
        if (k < nh && k > first) {
            if (r.sp < TRACE_STACK) stack.push(r.sp++, val[k], key[k]);
            else atomicOr(a.err, ERR_STACK);
        }
    }
    // a directly entered leaf always waits behind the parked one; only a
    // pop can bring a leaf to park
    if (first < nh) r.node = first ? val[1] : val[0];
    else advance(r, stack);
}

// Test the parked leaf, if any.
template <bool COUNT, class A>
__device__ __forceinline__ void leaf_step(const A& a, Ray& r, Stack& stack, uint32_t& visits, uint32_t& tests) {
    const int leaf = r.leaf;
    if (leaf == WIDE_EMPTY) return;
    r.steps++;
    if (COUNT) {
        visits++;
        tests++;
    }
    // one triangle = two aligned 32-byte sectors (v0 | index, e1) and (e2, pad)
    float4 p0, p1, p2, pad;
    ldg256(&a.tri[TRI_F4 * leaf], p0, p1);
    ldg256(&a.tri[TRI_F4 * leaf + 2], p2, pad);
    float t;
    bool fr;
    if (ray_tri(r.o, r.d, make_float3(p0.x, p0.y, p0.z), make_float3(p1.x, p1.y, p1.z),
                make_float3(p2.x, p2.y, p2.z), t, fr)) {
        const int idx = __float_as_int(p0.w);
        if (t < r.bt || (t == r.bt && idx < r.bidx)) {
            r.bt = t;
            r.bidx = idx;
            r.bfront = fr;
        }
    }
    r.leaf = WIDE_EMPTY;
    if (r.node != WIDE_EMPTY && r.node < 0) {
        r.leaf = ~r.node;
        advance(r, stack);
    }
}

// One warp iteration of the two-phase traversal for every lane (active or
// not: call it convergently): NODE_STEPS node steps, then the leaf phase if
// enough lanes wait on a parked leaf.  Two node steps per iteration halve
// the cost of the phase decision (three ballots) per node visit; measured on
// the 1M-triangle frame: 1 step 525 ms, 2 steps 497 ms, 3 steps 517 ms,
// 4 steps 499 ms.  Returns true for a lane whose ray finished.
constexpr int NODE_STEPS = 2;

// COUNT: visits / tests count this lane's node visits and triangle tests,
// leaf_slots the leaf rounds the warp ran (one or two per leaf phase).
template <bool COUNT, bool TEX, class A>
__device__ __forceinline__ bool warp_step(const A& a, Ray& r, Stack& stack, bool active, int leaf_min,
                                          uint32_t& visits, uint32_t& tests, uint32_t& leaf_slots) {
    if (active) {
#pragma unroll
        for (int i = 0; i < NODE_STEPS; i++) node_step<COUNT, TEX>(a, r, stack, visits);
    }
    const bool parked = active && r.leaf != WIDE_EMPTY;
    const bool blocked = parked && r.node < 0;             // cannot go on before its leaf
    const unsigned pm = __ballot_sync(0xFFFFFFFFu, parked);
    const unsigned bm = __ballot_sync(0xFFFFFFFFu, blocked);
    const unsigned im = __ballot_sync(0xFFFFFFFFu, active && r.node >= 0);
    if (pm && (__popc(pm) >= leaf_min || 2 * __popc(bm) >= leaf_min || im == 0)) {
        if (COUNT) leaf_slots++;
        if (parked) leaf_step<COUNT>(a, r, stack, visits, tests);
        // a lane whose next node was a leaf waiting behind the tested one has
        // parked it now and tests it in a second round of this phase (any
        // lane: measured slightly faster than waiting for several)
        const bool again = parked && r.leaf != WIDE_EMPTY;
        const unsigned am = __ballot_sync(0xFFFFFFFFu, again);
        if (am) {
            if (COUNT) leaf_slots++;
            if (again) leaf_step<COUNT>(a, r, stack, visits, tests);
        }
    }
    if (active) step_guard(a, r);
    return active && ray_done(r);
}

// L2 policy for data that streams past the tracer (the per-slot scratch of
// finished rays): evicted first, so that the BVH nodes and leaf triangles
// the traversal re-reads keep their place in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void red_min_stream(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("red.relaxed.gpu.global.min.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_stream(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// Commit of finished rays that share a texel slot (peers: the lanes of the
// same slot among those finishing now; lt: lanes below this one).  Vote:
// the minimum distance bits and the front | back << 16 hit counts.
// Nearest face: the minimum of (distance bits << 1 | back), ties -> front.
__device__ __forceinline__ void commit_ray(const Ray& r, bool nearest, unsigned peers, unsigned lt,
                                           uint32_t* ray_min, uint32_t* ray_cnt) {
    const bool hit = r.bidx != 0x7FFFFFFF;
    const uint32_t tbits = __float_as_uint(r.bt) & 0x7FFFFFFFu;
    if (nearest) {
        const uint32_t key = hit ? ((tbits << 1) | (r.bfront ? 0u : 1u)) : 0xFFFFFFFFu;
        const uint32_t mn = __reduce_min_sync(peers, key);
        if ((peers & lt) == 0 && mn != 0xFFFFFFFFu) red_min_stream(ray_min + r.slot, mn, l2_evict_first());
        return;
    }
    const uint32_t tb = hit ? tbits : 0x7F800000u;
    const uint32_t cv = hit ? (r.bfront ? 1u : 0x10000u) : 0u;
    const uint32_t mn = __reduce_min_sync(peers, tb);
    const uint32_t sum = __reduce_add_sync(peers, cv);
    if ((peers & lt) == 0) {
        const uint64_t pol = l2_evict_first();
        if (mn != 0x7F800000u) red_min_stream(ray_min + r.slot, mn, pol);
        if (sum) red_add_stream(ray_cnt + r.slot, sum, pol);
    }
}

// Eq. 1 for one texel slot after its rays committed: u_t = min(u, r_t) (the
// alpha decay was applied by the mask stage), counts += this frame's hits
// (saturating at 16 bits), f_t = +-u_t or c_t while no ray has hit; the
// slot's scratch is cleared for the next frame.
__device__ __forceinline__ void finalize_slot(const TraceArgs& a, uint64_t s) {
    // every access here streams (each slot and texel is touched once per
    // frame): cache-streaming loads and stores keep the BVH in L2
    const uint32_t parent = __ldcs(a.masked + (s >> 3));
    const uint32_t ch = (uint32_t)(s & 7);
    const uint32_t nc = (uint32_t)a.nc, nf = 2u * nc;
    const uint32_t pq = __umulhi(parent, a.nc_mag), pz = __umulhi(pq, a.nc_mag);
    const uint32_t px = parent - pq * nc, py = pq - pz * nc;
    const uint32_t texel = (2 * px + (ch & 1)) + nf * ((2 * py + ((ch >> 1) & 1)) + nf * (2 * pz + (ch >> 2)));
    if (a.nearest) {
        // Eq. 1's minimum over (u, this frame's nearest hit), keeping the face
        // of the smaller one (counts holds the face: 1 = back)
        const uint32_t km = __ldcs(a.ray_min + s);
        __stcs(a.ray_min + s, ray_min_none(true));
        const float u0 = __ldcs(a.accum + texel);
        const uint32_t kp =
            u0 == CUDART_INF_F ? 0xFFFFFFFFu : ((__float_as_uint(u0) << 1) | (__ldcs(a.counts + texel) & 1u));
        const uint32_t k = min(kp, km);
        if (k == 0xFFFFFFFFu) {
            __stcs(a.fine + texel, __ldcs(a.coarse + parent));
            return;
        }
        const float u = __uint_as_float(k >> 1);
        __stcs(a.accum + texel, u);
        __stcs(a.counts + texel, k & 1u);
        __stcs(a.fine + texel, (k & 1u) ? -u : u);
        return;
    }
    const float rmin = __uint_as_float(__ldcs(a.ray_min + s));
    const uint32_t cv = __ldcs(a.ray_cnt + s);
    __stcs(a.ray_min + s, ray_min_none(false));
    __stcs(a.ray_cnt + s, 0u);
    const float u = fminf(__ldcs(a.accum + texel), rmin);
    const uint32_t cw = __ldcs(a.counts + texel);
    const uint32_t f = min((cw & 0xFFFFu) + (cv & 0xFFFFu), 0xFFFFu);
    const uint32_t b = min((cw >> 16) + (cv >> 16), 0xFFFFu);
    __stcs(a.accum + texel, u);
    __stcs(a.counts + texel, f | (b << 16));
    const float mag = u == CUDART_INF_F ? __ldcs(a.coarse + parent) : u;
    __stcs(a.fine + texel, b > f ? -mag : mag);
}

}  // namespace dev
}  // namespace rtsdf
