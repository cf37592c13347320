// Sec. 2.2 -- ray tracing of the masked fine texels with temporal
// accumulation (Eq. 1) and the front/back sign vote.
//
// Each masked coarse voxel contributes its 8 fine children ("texel slots");
// each slot casts R rays, so the frame's work is a flat list of
// 8 * masked * R ray ids (consecutive ids share a texel).  Per ray:
//   * the direction comes from Philox-4x32-10 (Salmon et al., SC'11) with
//     counter (draw, ray, frame, texel) and key (seed lo, seed hi), mapped to
//     the sphere by Marsaglia's (1972) rejection method -- integer accept
//     test, fp32 map, so every direction is bit-reproducible;
//   * the closest hit comes from a stack traversal of the 4-wide BVH (one
//     128-byte node fetch tests four child boxes; the nearest hit child is
//     entered next, the others pushed farthest-first with their entry
//     distance and skipped on pop once they cannot hold a closer hit),
//     leaves tested with Moller-Trumbore in fp32 with the operation
//     order written out (explicit fma / rounding intrinsics); equal
//     distances keep the smaller original triangle index.
// Rays of very different lengths would leave most lanes of a lock-step warp
// idle, so warps are persistent and refill idle lanes with new ray ids from
// a warp-local chunk once enough lanes are idle.  The traversal runs in two
// phases (a lane parks the leaf it reaches and keeps descending; the warp
// tests triangles when enough lanes hold a parked leaf), two node steps per
// phase decision.  A finished ray commits its distance (atomicMin on the
// float bits, t >= 0) and its front/back hit into per-slot scratch with
// warp-aggregated atomics; k_trace_finalize then applies Eq. 1 per texel:
// u_t = min(u, r_t) (the alpha decay was applied by the mask kernel), the
// counts, and f_t = +-u_t (c_t while no ray has hit), negative when back
// hits outnumber front hits.  In the nearest-face sign mode a ray starts
// with the texel's u as its best hit and commits (t, face) as one key.
#include <math_constants.h>

#include "internal.cuh"
#include "trace_dev.cuh"

namespace rtsdf {
namespace {

using namespace dev;

// Persistent warps: each lane traces one ray at a time and takes a new one
// as soon as it finishes (from a warp-local chunk of consecutive ray ids, so
// the lanes of a warp mostly share a texel and its origin).  Finished rays
// commit (min distance, front/back) per texel slot with warp-aggregated
// atomics; k_trace_finalize then applies Eq. 1 per texel.
template <bool COUNT, bool TEX>
__global__ void __launch_bounds__(TRACE_THREADS, 8) k_trace(TraceArgs a) {
    uint32_t n_visits = 0, n_tests = 0, n_rays = 0;
    uint32_t n_slots = 0, n_leaf_slots = 0;   // COUNT: traversal iterations, leaf phases run
    const uint64_t total = (uint64_t)(*a.count) * 8u * (uint64_t)a.rays;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    // traversal stack: the first SMEM_STACK (node, distance) entries in shared
    // memory laid out [entry][thread], deeper entries in local memory
    __shared__ int2 s_stack[SMEM_STACK][TRACE_THREADS];
    int2 deep[TRACE_STACK - SMEM_STACK];
    Stack stk{&s_stack[0][threadIdx.x], deep};
    // per-warp chunk of ray ids, kept in shared memory (read only at refills)
    // so that the traversal loop keeps its registers
    __shared__ unsigned long long s_cnext[TRACE_THREADS / 32], s_cend[TRACE_THREADS / 32];
    const unsigned wi = threadIdx.x >> 5;
    if (lane == 0) s_cnext[wi] = s_cend[wi] = 0;
    __syncwarp();
    Ray r;
    bool active = false;
    bool exhausted = false;                    // warp-uniform
    for (;;) {
        // hand out rays to idle lanes
        unsigned idle = __ballot_sync(0xFFFFFFFFu, !active);
        while (idle && !exhausted) {
            uint64_t cn = s_cnext[wi];
            if (cn == s_cend[wi]) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(a.next_ray, (unsigned long long)a.ray_chunk);
                b = __shfl_sync(0xFFFFFFFFu, b, 0);
                if (b >= total) {
                    exhausted = true;
                    break;
                }
                cn = b;
                __syncwarp();
                if (lane == 0) s_cend[wi] = min((uint64_t)b + (uint64_t)a.ray_chunk, total);
                __syncwarp();
            }
            const uint32_t avail = (uint32_t)(s_cend[wi] - cn);
            const uint32_t want = __popc(idle);
            const uint32_t take = min(avail, want);
            if (!active) {
                const uint32_t rank = __popc(idle & lt);
                if (rank < take) {
                    setup_ray(a, cn + rank, r);
                    active = true;
                    if (COUNT) n_rays++;
                }
            }
            __syncwarp();
            if (lane == 0) s_cnext[wi] = cn + take;
            __syncwarp();
            idle = __ballot_sync(0xFFFFFFFFu, !active);
        }
        if (__ballot_sync(0xFFFFFFFFu, active) == 0) break;
        // trace until enough lanes are idle to be worth a refill
        for (;;) {
            const bool done = warp_step<COUNT, TEX>(a, r, stk, active, a.leaf_min, n_visits, n_tests, n_leaf_slots);
            if (COUNT) n_slots += NODE_STEPS;   // lane slots of the node steps
            const unsigned fin = __ballot_sync(0xFFFFFFFFu, done);
            if (fin && done) {
                const unsigned peers = __match_any_sync(fin, r.slot);
                commit_ray(r, a.nearest != 0, peers, lt, a.ray_min, a.ray_cnt);
                active = false;
            }
            const unsigned act = __ballot_sync(0xFFFFFFFFu, active);
            if (act == 0) break;
            if (!exhausted && (32 - __popc(act)) >= a.refill_min) break;
        }
    }
    if (COUNT) {
        // summed over the warp's lanes, the iteration counts become lane slots
        unsigned long long rr = n_rays, v = n_visits, t = n_tests, sl = n_slots, ls = n_leaf_slots;
        for (int off = 16; off >= 1; off >>= 1) {
            rr += __shfl_xor_sync(0xFFFFFFFFu, rr, off);
            v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
            t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
            sl += __shfl_xor_sync(0xFFFFFFFFu, sl, off);
            ls += __shfl_xor_sync(0xFFFFFFFFu, ls, off);
        }
        if (lane == 0) {
            atomicAdd(&a.counters->rays, rr);
            atomicAdd(&a.counters->visits, v);
            atomicAdd(&a.counters->tests, t);
            atomicAdd(&a.counters->slots, sl);
            atomicAdd(&a.counters->leaf_slots, ls);
        }
    }
}

// Eq. 1 per traced texel slot (see finalize_slot): a grid-stride loop over
// the frame's slots (8 per masked voxel, a count known only on the device).
__global__ void __launch_bounds__(256) k_trace_finalize(TraceArgs a) {
    const uint64_t n = (uint64_t)(*a.count) * 8u;
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += stride) finalize_slot(a, s);
}

}  // namespace

cudaError_t trace_occupancy(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_trace<false, true>, TRACE_THREADS, 0);
}

cudaError_t launch_trace(rtsdf_ctx* c, int rays, int frame) {
    TraceArgs a;
    a.masked = c->masked;
    a.count = c->d_masked_count;
    a.nc = c->nc;
    a.rays = rays;
    int lg = 0;
    while ((1 << lg) < rays) lg++;
    a.log2_rays = lg;
    a.key0 = (uint32_t)c->cfg.seed;
    a.key1 = (uint32_t)(c->cfg.seed >> 32);
    a.frame = (uint32_t)frame;
    a.bx = c->cfg.bmin[0];
    a.by = c->cfg.bmin[1];
    a.bz = c->cfg.bmin[2];
    a.hf = c->hf;
    a.wide = c->bvh.wide;
    a.wtex = texture_fetch_on() ? c->bvh.wtex : 0;
    a.tri = c->bvh.tri;
    a.nt = c->bvh.nt;
    a.coarse = c->coarse;
    a.accum = c->accum;
    a.counts = c->counts;
    a.fine = c->fine;
    a.err = c->d_err;
    a.counters = c->d_counters;
    a.ray_min = c->ray_min;
    a.ray_cnt = c->ray_cnt;
    a.next_ray = c->d_next_ray;
    a.refill_min = c->tune.refill_min;
    a.ray_chunk = c->tune.ray_chunk;
    a.leaf_min = c->tune.leaf_min;
    a.nc_mag = (uint32_t)((0x100000000ull + (unsigned long long)c->nc - 1) / (unsigned long long)c->nc);
    a.nearest = c->sign_mode == RTSDF_SIGN_NEAREST;
    cudaError_t e = cudaMemsetAsync(c->d_next_ray, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        if (a.wtex) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<false, true>, TRACE_THREADS, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<false, false>, TRACE_THREADS, 0);
        if (per_sm < 1) per_sm = 4;
        const int use = (c->tune.trace_blocks_per_sm > 0 && c->tune.trace_blocks_per_sm < per_sm)
                            ? c->tune.trace_blocks_per_sm : per_sm;
        c->trace_grid = (unsigned)(sms > 0 ? sms : 132) * (unsigned)use;
    }
    // the texture path when the node texture exists (plain loads otherwise)
    if (a.wtex) {
        if (c->counting) RTSDF_LAUNCH(c, (k_trace<true, true>), c->trace_grid, TRACE_THREADS, 0, a);
        else RTSDF_LAUNCH(c, (k_trace<false, true>), c->trace_grid, TRACE_THREADS, 0, a);
    } else {
        if (c->counting) RTSDF_LAUNCH(c, (k_trace<true, false>), c->trace_grid, TRACE_THREADS, 0, a);
        else RTSDF_LAUNCH(c, (k_trace<false, false>), c->trace_grid, TRACE_THREADS, 0, a);
    }
    // the slot count is on the device: enough blocks to fill every SM
    // (8 x 256 threads each), capped by the largest possible slot count
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const uint64_t most = (8 * (uint64_t)c->nc3 + 255) / 256;
        const uint64_t want = (uint64_t)(sms > 0 ? sms : 132) * 8u;
        RTSDF_LAUNCH(c, k_trace_finalize, (unsigned)(most < want ? most : want), 256, 0, a);
    }
    return cudaGetLastError();
}

}  // namespace rtsdf
