// Batched form: many independent scenes of uneven grid and mesh size, the
// whole per-frame pipeline (clear, voxelize, jump flood, mask, trace, Eq. 1
// finalize) for all of them in ONE persistent cooperative launch, replayed
// from a CUDA graph -- or, with split_trace, that launch up to the mask and
// the trace and finalize as two more launches in the same graph: the
// persistent launch's register budget (64, 8 blocks per SM) is set by its
// other stages, while the traversal, bound by instruction issue, runs 4 %
// faster at the tracer's own 9 blocks per SM.
//
// Work of every stage is flattened over the scenes through prefix sums (a
// thread finds its scene by binary search), so small scenes do not leave
// the GPU idle and no per-scene launch or tail is paid.  Stages are separated
// by a grid-wide barrier; the tracer fetches rays dynamically across all
// scenes.  The arithmetic is the per-scene path's own (vox_dev.cuh,
// jfa_dev.cuh, trace_dev.cuh), so each scene's result equals a plain
// per-scene frame bit for bit.
//
// The barrier is an arrival counter plus a generation word.  Its waits are
// bounded: after BARRIER_SPINS polls a block records ERR_TIMEOUT, raises a
// shared abort flag and the whole kernel returns (rtsdf_batch_sync then
// reports RTSDF_E_TIMEOUT); the cooperative launch guarantees that all
// blocks are resident, so the bound only guards against a broken launch.
#include <math.h>
#include <math_constants.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"
#include "jfa_dev.cuh"
#include "trace_dev.cuh"
#include "vox_dev.cuh"

namespace rtsdf {
namespace {

using namespace dev;

constexpr int MAX_BATCH = 256;
// minimum resident blocks per SM the compiler must allow (register budget
// 65536 / (128 x this) per thread)
#ifndef BATCH_BLOCKS_PER_SM
#define BATCH_BLOCKS_PER_SM 8
#endif
constexpr uint32_t BARRIER_SPINS = 1u << 27;   // default polls (>= 64 ns each): several seconds

struct SceneDesc {
    TraceArgs t;              // tracer fields (rays / frame filled in per frame)
    const int32_t* q;         // quantised vertices
    const int32_t* tris;
    long long n_tris;
    uint32_t* seeds[2];
    float hc, beta_h, beta_vox, alpha;
    int passes;
    int wide_off, tri_off;    // this scene's nodes / leaves in the concatenated BVH
    uint32_t nmag;            // ceil(2^32 / nc): q = umulhi(v, nmag) = v / nc for v < 2^24
};

struct BatchParams {
    uint32_t frame;
    int rays, log2_rays;
    float d_vox;
};

struct BvhRef {
    const WNode* wide;
    cudaTextureObject_t wtex;   // the same nodes as int4 texels (used by the TEX trace)
    const float4* tri;
    long long nt;
    uint32_t* err;
};

struct BatchArgs {
    const SceneDesc* sc;
    int ns;
    const BatchParams* params;
    const unsigned long long* vox_prefix;   // [ns + 1] coarse voxels
    const unsigned long long* tri_prefix;   // [ns + 1] triangles
    int max_passes;
    int2* big_list;                         // (scene, triangle) of large triangles
    uint32_t* big_count;
    unsigned long long* next_ray;
    uint32_t* bar_count;
    uint32_t* bar_gen;
    uint32_t* abort;
    uint32_t* err;
    int refill_min;
    int ray_chunk;
    int leaf_min;
    uint32_t spins;
    unsigned long long* stamps;   // [8] global timer at the stage boundaries (block 0)
    BvhRef bvh;               // every scene's BVH in one array (child ids rebased)
    int split;                // 1: trace and finalize run as two launches after the pipeline launch
    int phase;                // split form: 1 = stages 0-2 (the jump flood follows as launches of its
                              // own), 2 = stage 4 on; 0 = the whole frame in one launch
    const uint32_t* jfa_blocks;   // split jump flood: [max_passes][ns + 1] prefix over scenes of their blocks
    unsigned long long* ray_prefix;   // [ns + 1] split form: ray prefix over scenes, written after the mask
    uint32_t* fin_done;       // split finalize: blocks done (the last one stamps the frame's end)
};

__device__ __forceinline__ int find_scene(const unsigned long long* prefix, int ns, unsigned long long g) {
    int lo = 0, hi = ns - 1;   // largest s with prefix[s] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void write_stamp(const BatchArgs& b, int k) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    b.stamps[k] = t;
}

__device__ __forceinline__ void stamp(const BatchArgs& b, int k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) write_stamp(b, k);
}

__device__ bool grid_barrier(const BatchArgs& b) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* gen = b.bar_gen;
        volatile uint32_t* abort = b.abort;
        const uint32_t g0 = *gen;
        __threadfence();
        if (atomicAdd(b.bar_count, 1u) + 1u == gridDim.x) {
            *b.bar_count = 0u;
            __threadfence();
            atomicAdd(b.bar_gen, 1u);
        } else {
            for (uint32_t it = 0; *gen == g0 && *abort == 0u; it++) {
                if (it > b.spins) {
                    atomicOr(b.err, ERR_TIMEOUT);
                    atomicExch(b.abort, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = *abort == 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

// Stages 1 and 2 of the batched frame, out of line: the 13-axis overlap
// setup needs many registers, which would otherwise be reserved across the
// whole kernel (and spill in the tracer loop).
__device__ __noinline__ void batch_voxelize_small(const BatchArgs& b, uint64_t tid, uint64_t nthr) {
    const int ns = b.ns;
    const unsigned long long total_tris = b.tri_prefix[ns];
    for (uint64_t g = tid; g < total_tris; g += nthr) {
        const int s = find_scene(b.tri_prefix, ns, g);
        const SceneDesc& d = b.sc[s];
        const long long t = (long long)(g - b.tri_prefix[s]);
        const int n = d.t.nc;
        TriAxes ax;
        setup(d.q, d.tris, t, n, ax);
        const int cx = ax.hi[0] - ax.lo[0] + 1, cy = ax.hi[1] - ax.lo[1] + 1, cz = ax.hi[2] - ax.lo[2] + 1;
        if (cx <= 0 || cy <= 0 || cz <= 0) continue;
        if ((long long)cx * cy * cz > SMALL_MAX) {
            b.big_list[atomicAdd(b.big_count, 1u)] = make_int2(s, (int)t);
            continue;
        }
        for (int z = ax.lo[2]; z <= ax.hi[2]; z++)
            for (int y = ax.lo[1]; y <= ax.hi[1]; y++)
                for (int x = ax.lo[0]; x <= ax.hi[0]; x++)
                    if (overlaps(ax, x, y, z)) d.seeds[0][x + (size_t)n * (y + (size_t)n * z)] = pack_seed(x, y, z);
    }
}

__device__ __noinline__ void batch_voxelize_big(const BatchArgs& b) {
    {
        const uint32_t nb = *(volatile uint32_t*)b.big_count;
        for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
            const int2 it = b.big_list[i];
            const SceneDesc& d = b.sc[it.x];
            const int n = d.t.nc;
            TriAxes ax;
            setup(d.q, d.tris, it.y, n, ax);
            const int cx = ax.hi[0] - ax.lo[0] + 1, cy = ax.hi[1] - ax.lo[1] + 1, cz = ax.hi[2] - ax.lo[2] + 1;
            const long long tot = (long long)cx * cy * cz;
            for (long long v = threadIdx.x; v < tot; v += blockDim.x) {
                const int x = ax.lo[0] + (int)(v % cx), y = ax.lo[1] + (int)((v / cx) % cy);
                const int z = ax.lo[2] + (int)(v / ((long long)cx * cy));
                if (overlaps(ax, x, y, z)) d.seeds[0][x + (size_t)n * (y + (size_t)n * z)] = pack_seed(x, y, z);
            }
        }
    }
}

// Jump-flood pass p of every scene that has one, as one grid-stride loop
// over all scenes' voxels (voxel prefix vp), so that small scenes do not
// leave most threads idle; a thread's voxel index only grows, so its scene
// index only moves forward.  Not inlined: the 27 candidates' registers then
// do not shape the register allocation of the whole persistent kernel (the
// trace stage above all).
__device__ __noinline__ void batch_jfa_pass(const BatchArgs& b, const unsigned long long* vp, int ns, int p,
                                            uint64_t tid, uint64_t nthr) {
    const unsigned long long total = vp[ns];
    int s = -1;
    unsigned long long lo = 0, hi = 0;
    for (unsigned long long g = tid; g < total; g += nthr) {
        if (g >= hi) {
            do s++;
            while (vp[s + 1] <= g);
            lo = vp[s];
            hi = vp[s + 1];
        }
        const SceneDesc& d = b.sc[s];
        const int L = d.passes;
        if (p >= L) {          // this scene has no pass p: skip its voxels
            g = hi - 1 - ((hi - 1 - g) % nthr);
            continue;
        }
        const uint32_t n = (uint32_t)d.t.nc, mag = d.nmag;
        const uint32_t v = (uint32_t)(g - lo);
        const uint32_t vq = __umulhi(v, mag), z = __umulhi(vq, mag);
        const int x = (int)(v - vq * n), y = (int)(vq - z * n);
        const int k = 1 << (L - 1 - p);
        const uint32_t* in = d.seeds[p & 1];
        uint32_t* out = d.seeds[(p + 1) & 1];
        float* coarse = const_cast<float*>(d.t.coarse);
        if (p == L - 1) jfa_voxel<true, false>(in, out, (int)n, k, x, y, (int)z, coarse, d.hc, d.beta_h);
        else jfa_voxel<false, false>(in, out, (int)n, k, x, y, (int)z, coarse, d.hc, d.beta_h);
    }
}

// Split form of stage 3: jump-flood pass p of every scene that has one as
// one launch of the per-scene z-blocked pass (dev::jfa_zblock_column, T = 8)
// over all scenes' columns: blocks of 32 x 4 threads, a scene's blocks
// consecutive (jfa_blocks row p: prefix over scenes of their block counts,
// 0 for a scene without pass p).  Inside the pipeline launch the pass would
// have that launch's register budget, which rules out the register-blocked
// columns.  Skips its work when the pipeline launch gave up at a barrier.
__global__ void __launch_bounds__(128, 4) k_batch_jfa(BatchArgs b, int p) {
    if (*(volatile const uint32_t*)b.abort) return;
    const uint32_t* pre = b.jfa_blocks + (size_t)p * (size_t)(b.ns + 1);
    const uint32_t blk = blockIdx.x;
    int lo = 0, hi = b.ns - 1;   // largest s with pre[s] <= blk (a scene without blocks is skipped)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    const SceneDesc& d = b.sc[lo];
    const int n = d.t.nc, L = d.passes;
    const int k = 1 << (L - 1 - p);
    const uint32_t nbx = ((uint32_t)n + 31u) / 32u, nby = ((uint32_t)n + 3u) / 4u;
    uint32_t local = blk - pre[lo];
    const uint32_t bx = local % nbx;
    local /= nbx;
    const uint32_t by = local % nby, bz = local / nby;
    const int x = (int)(bx * 32u + threadIdx.x), y = (int)(by * 4u + threadIdx.y);
    if (x >= n || y >= n) return;
    const int rz = (int)(bz % (uint32_t)k), g = (int)(bz / (uint32_t)k);
    const uint32_t* in = d.seeds[p & 1];
    uint32_t* out = d.seeds[(p + 1) & 1];
    float* coarse = const_cast<float*>(d.t.coarse);
    if (p == L - 1) dev::jfa_zblock_column<true, 8>(in, out, n, k, x, y, rz, g, coarse, d.hc, d.beta_h);
    else dev::jfa_zblock_column<false, 8>(in, out, n, k, x, y, rz, g, coarse, d.hc, d.beta_h);
}

// Ray prefix over scenes (8 texel slots per masked voxel, `rays` rays
// each), in shared memory; every thread of the block returns with it.
__device__ __forceinline__ void batch_ray_prefix(const BatchArgs& b, unsigned long long* s_rp, int ns, int rays) {
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int s = 0; s < ns; s++) {
            s_rp[s] = acc;
            acc += (unsigned long long)(*(volatile const uint32_t*)b.sc[s].t.count) * 8ull * (unsigned long long)rays;
        }
        s_rp[ns] = acc;
    }
    __syncthreads();
}

// Stage 5: all scenes' rays from one dynamic counter (the per-scene
// tracer's persistent-warp traversal; each lane remembers its ray's scene).
// TEX: node fetches split between the load and texture pipes.
template <bool TEX>
__device__ __forceinline__ void batch_trace_rays(const BatchArgs& b, const unsigned long long* s_rp, int ns) {
    __shared__ int2 s_stack[SMEM_STACK][TRACE_THREADS];
    // per-warp chunk state, kept in shared memory (read only at refills) so
    // that the traversal loop keeps its registers
    __shared__ unsigned long long s_cnext[TRACE_THREADS / 32], s_cend[TRACE_THREADS / 32];
    __shared__ unsigned long long s_csend[TRACE_THREADS / 32];
    __shared__ int s_cscene[TRACE_THREADS / 32];
    __shared__ uint8_t s_scene[TRACE_THREADS];   // scene of each lane's ray (< MAX_BATCH; read at setup and commit)
    const unsigned lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int2 deep[TRACE_STACK - SMEM_STACK];
    Stack stk{&s_stack[0][threadIdx.x], deep};
    Ray r;
    bool active = false;
    bool exhausted = false;
    uint32_t dummy_v = 0, dummy_t = 0, dummy_l = 0;
    if (lane == 0) s_cnext[wi] = s_cend[wi] = 0;
    __syncwarp();
    for (;;) {
        unsigned idle = __ballot_sync(0xFFFFFFFFu, !active);
        while (idle && !exhausted) {
            unsigned long long cn = s_cnext[wi];
            if (cn == s_cend[wi]) {
                unsigned long long c0 = 0;
                if (lane == 0) c0 = atomicAdd(b.next_ray, (unsigned long long)b.ray_chunk);
                c0 = __shfl_sync(0xFFFFFFFFu, c0, 0);
                const unsigned long long total = s_rp[ns];
                if (c0 >= total) {
                    exhausted = true;
                    break;
                }
                cn = c0;
                __syncwarp();
                if (lane == 0) {
                    // scene of the chunk's first ray and where that scene ends
                    const int cs = find_scene(s_rp, ns, c0);
                    s_cscene[wi] = cs;
                    s_csend[wi] = s_rp[cs + 1];
                    s_cend[wi] = min(c0 + (unsigned long long)b.ray_chunk, total);
                }
                __syncwarp();
            }
            const uint32_t avail = (uint32_t)(s_cend[wi] - cn);
            const uint32_t want = __popc(idle);
            const uint32_t take = min(avail, want);
            if (!active) {
                const uint32_t rank = __popc(idle & lt);
                if (rank < take) {
                    const unsigned long long g = cn + rank;
                    const int scene = g < s_csend[wi] ? s_cscene[wi] : find_scene(s_rp, ns, g);
                    s_scene[threadIdx.x] = (uint8_t)scene;
                    const TraceArgs& ta = b.sc[scene].t;
                    setup_ray(ta, g - s_rp[scene], r);
                    // enter the scene's root in the concatenated tree
                    const SceneDesc& sd = b.sc[scene];
                    r.node = ta.nt > 1 ? sd.wide_off : WIDE_EMPTY;
                    r.leaf = ta.nt == 1 ? sd.tri_off : WIDE_EMPTY;
                    active = true;
                }
            }
            __syncwarp();
            if (lane == 0) s_cnext[wi] = cn + take;
            __syncwarp();
            idle = __ballot_sync(0xFFFFFFFFu, !active);
        }
        if (__ballot_sync(0xFFFFFFFFu, active) == 0) break;
        for (;;) {
            const bool done = warp_step<false, TEX>(b.bvh, r, stk, active, b.leaf_min, dummy_v, dummy_t, dummy_l);
            const unsigned fin = __ballot_sync(0xFFFFFFFFu, done);
            if (fin && done) {
                const int scene = (int)s_scene[threadIdx.x];
                const unsigned long long key = ((unsigned long long)scene << 32) | r.slot;
                const unsigned peers = __match_any_sync(fin, key);
                const TraceArgs& st = b.sc[scene].t;
                commit_ray(r, st.nearest != 0, peers, lt, st.ray_min, st.ray_cnt);
                active = false;
            }
            const unsigned act = __ballot_sync(0xFFFFFFFFu, active);
            if (act == 0) break;
            if (!exhausted && (32 - __popc(act)) >= b.refill_min) break;
        }
    }
}

// Stage 6: one grid-stride loop over every scene's slots (slot prefix = ray
// prefix >> log2 rays); a thread's slot index only grows, so its scene index
// only moves forward.
__device__ __forceinline__ void batch_finalize(const BatchArgs& b, const unsigned long long* s_rp, int ns, int lg) {
    const unsigned long long stot = s_rp[ns] >> lg;
    int sc = -1;
    unsigned long long lo = 0, hi = 0;   // slot range of scene sc
    const TraceArgs* ta = nullptr;
    const unsigned long long ftid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long fnthr = gridDim.x * (unsigned long long)blockDim.x;
    for (unsigned long long g = ftid; g < stot; g += fnthr) {
        if (g >= hi) {
            do sc++;
            while ((s_rp[sc + 1] >> lg) <= g);
            lo = s_rp[sc] >> lg;
            hi = s_rp[sc + 1] >> lg;
            ta = &b.sc[sc].t;
        }
        finalize_slot(*ta, g - lo);
    }
}

__global__ void __launch_bounds__(TRACE_THREADS, BATCH_BLOCKS_PER_SM) k_batch_frame(BatchArgs b) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nthr = gridDim.x * (uint64_t)blockDim.x;
    // the frame's parameters live in shared memory, not in registers that
    // would stay allocated through the trace stage
    __shared__ BatchParams P;
    const int ns = b.ns;
    if (b.phase != 2) stamp(b, 0);
    // prefix over scenes: voxels in stages 0-4, rays in stages 5-6
    __shared__ unsigned long long s_prefix[MAX_BATCH + 1];
    unsigned long long* s_vp = s_prefix;
    if (threadIdx.x == 0) P = *b.params;
    for (int i = threadIdx.x; i <= ns; i += blockDim.x) s_vp[i] = b.vox_prefix[i];
    __syncthreads();
    if (b.phase == 2 && *(volatile const uint32_t*)b.abort) return;
    if (b.phase != 2) {   // stages 0-3 (phase 2 starts after the flood launches)
        // ---- stage 0: clear the seed grids and the per-scene counters
        for (int s = 0; s < ns; s++) {
            const uint64_t n3 = s_vp[s + 1] - s_vp[s];
            uint32_t* sd = b.sc[s].seeds[0];
            for (uint64_t g = tid; g < n3; g += nthr) sd[g] = SEED_EMPTY;
        }
        for (uint64_t s = tid; s < (uint64_t)ns; s += nthr) {
            // the frame's ray parameters go into each scene's tracer fields, so
            // that the trace stage reads them in place (no copy of the fields)
            TraceArgs& t = const_cast<SceneDesc&>(b.sc[s]).t;
            *const_cast<uint32_t*>(t.count) = 0u;
            t.rays = P.rays;
            t.log2_rays = P.log2_rays;
            t.frame = P.frame;
        }
        if (tid == 0) {
            *b.big_count = 0u;
            *b.next_ray = 0ull;
        }
        if (!grid_barrier(b)) return;
        stamp(b, 1);

        // ---- stage 1: voxelize (small triangles inline, large ones listed)
        batch_voxelize_small(b, tid, nthr);
        if (!grid_barrier(b)) return;
        stamp(b, 2);

        // ---- stage 2: large triangles, one block each
        batch_voxelize_big(b);
        if (!grid_barrier(b)) return;
        stamp(b, 3);
        if (b.phase == 1) return;   // the jump flood follows as launches of its own (k_batch_jfa)

        // ---- stage 3: jump flooding, pass p of every scene that has one
        for (int p = 0; p < b.max_passes; p++) {
            batch_jfa_pass(b, s_vp, ns, p, tid, nthr);
            if (!grid_barrier(b)) return;
        }
    }   // stages 0-3
    // scenes without jump steps (N = 1): coarse value straight from the seed
    for (uint64_t s = tid; s < (uint64_t)ns; s += nthr) {
        const SceneDesc& d = b.sc[s];
        if (d.passes == 0) {
            const uint32_t sv = d.seeds[0][0];
            const_cast<float*>(d.t.coarse)[0] = coarse_value(sv, seed_d2(sv, 0u, 0u), d.hc, d.beta_h);
        }
    }
    if (!grid_barrier(b)) return;
    stamp(b, 4);

    // ---- stage 4: near-surface mask, fill, Eq. 1 decay (static scenes: no reset)
    {
        const unsigned lane = threadIdx.x & 31;
        const uint32_t warp0 = (uint32_t)(tid - lane);
        for (int s = 0; s < ns; s++) {
            const SceneDesc& dg = b.sc[s];
            const uint32_t n = (uint32_t)dg.t.nc, mag = dg.nmag, n3 = n * n * n;
            if (warp0 >= n3) continue;
            // local copies: stores through the grid pointers below could
            // otherwise alias the descriptor and force reloads
            const uint32_t* seeds_fin = dg.seeds[dg.passes & 1];
            const float* coarse = dg.t.coarse;
            float* accum = dg.t.accum;
            uint32_t* counts = dg.t.counts;
            float* fine = dg.t.fine;
            uint32_t* list = const_cast<uint32_t*>(dg.t.masked);
            uint32_t* count = const_cast<uint32_t*>(dg.t.count);
            const float alpha = dg.alpha;
            const double sdv = (double)P.d_vox + (double)dg.beta_vox;
            const long long T = sdv < 0 ? -1 : (long long)floor(sdv * sdv);
            const uint32_t nf = 2 * n;
            for (uint32_t base = warp0; base < n3; base += (uint32_t)nthr) {
                const uint32_t v = base + lane;
                const bool valid = v < n3;
                bool masked = false;
                if (valid) {
                    const uint32_t vq = __umulhi(v, mag), z = __umulhi(vq, mag);
                    const int x = (int)(v - vq * n), y = (int)(vq - z * n);
                    const uint32_t sv = seeds_fin[v];
                    if (sv != SEED_EMPTY) {
                        const int dx = (int)(sv & 0xFF) - x, dy = (int)((sv >> 8) & 0xFF) - y;
                        const int dz = (int)((sv >> 16) & 0xFF) - (int)z;
                        masked = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz <= T;
                    }
                    const float c = coarse[v];
                    for (int cz = 0; cz < 2; cz++)
                        for (int cy = 0; cy < 2; cy++)
                            for (int cx = 0; cx < 2; cx++) {
                                const size_t j = (size_t)(2 * x + cx) +
                                                 (size_t)nf * ((size_t)(2 * y + cy) + (size_t)nf * (2 * z + cz));
                                const float u = accum[j];
                                if (!masked) {
                                    fine[j] = c;
                                    if (u != CUDART_INF_F) {
                                        accum[j] = CUDART_INF_F;
                                        counts[j] = 0u;
                                    }
                                } else if (alpha != 1.f) {
                                    float un = u;
                                    if (alpha == 0.f) un = c;
                                    else if (u != CUDART_INF_F)
                                        un = __fadd_rn(__fmul_rn(alpha, u), __fmul_rn(1.f - alpha, c));
                                    if (un != u) accum[j] = un;
                                }
                            }
                }
                // warp-aggregated append
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, masked);
                if (bal) {
                    const int leader = __ffs(bal) - 1;
                    uint32_t slot0 = 0;
                    if ((int)lane == leader) slot0 = atomicAdd(count, (uint32_t)__popc(bal));
                    slot0 = __shfl_sync(0xFFFFFFFFu, slot0, leader);
                    if (masked) list[slot0 + __popc(bal & ((1u << lane) - 1u))] = v;
                }
            }
        }
    }
    if (!grid_barrier(b)) return;
    stamp(b, 5);

    if (b.split) {
        // trace and finalize follow as launches of their own; they read the
        // ray prefix from global memory
        if (blockIdx.x == 0) {
            batch_ray_prefix(b, s_prefix, ns, P.rays);
            for (int i = threadIdx.x; i <= ns; i += blockDim.x) b.ray_prefix[i] = s_prefix[i];
        }
        return;
    }

    // ---- stage 5: trace all scenes' rays with dynamic fetch
    unsigned long long* s_rp = s_prefix;
    __syncthreads();   // every thread is done with the voxel prefix
    batch_ray_prefix(b, s_rp, ns, P.rays);
    batch_trace_rays<false>(b, s_rp, ns);
    if (!grid_barrier(b)) return;
    stamp(b, 6);

    // ---- stage 6: Eq. 1 finalize of every traced texel slot
    batch_finalize(b, s_rp, ns, P.log2_rays);
    grid_barrier(b);
    stamp(b, 7);
}

// Split form of stages 5 and 6: the trace as its own persistent launch,
// sized and register-bounded like the per-scene tracer (its occupancy sets
// its speed: the traversal is issue bound and hides latency with warps),
// then the finalize; both follow the pipeline launch on the stream and skip
// their work when that launch gave up at a barrier.
// (The bound asks for 8 resident blocks, i.e. at most 64 registers, as the
// per-scene tracer's does; the kernel compiles to 56 and runs 9 blocks per
// SM.  Asking for 9 forces 55 registers and code that issues 4 % more
// instructions per ray.)
#ifndef BATCH_TRACE_BLOCKS_PER_SM
#define BATCH_TRACE_BLOCKS_PER_SM 8
#endif

template <bool TEX>
__global__ void __launch_bounds__(TRACE_THREADS, BATCH_TRACE_BLOCKS_PER_SM) k_batch_trace(BatchArgs b) {
    if (*(volatile const uint32_t*)b.abort) return;
    batch_trace_rays<TEX>(b, b.ray_prefix, b.ns);
}

__global__ void __launch_bounds__(256) k_batch_finalize(BatchArgs b) {
    if (*(volatile const uint32_t*)b.abort) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) write_stamp(b, 6);   // the trace launch has ended
    batch_finalize(b, b.ray_prefix, b.ns, b.params->log2_rays);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(b.fin_done, 1u) == gridDim.x - 1) write_stamp(b, 7);   // the last block out
    }
}

// Copy one scene's 4-wide nodes into the concatenated array, rebasing child
// ids (internal by the scene's node offset, leaves by its leaf offset).
__global__ void k_rebase_nodes(const WNode* __restrict__ src, WNode* __restrict__ dst, int64_t n, int wide_off,
                               int tri_off) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    WNode w = src[i];
    int* ch = &w.child.x;
    for (int k = 0; k < 4; k++) {
        if (ch[k] == WIDE_EMPTY) continue;
        ch[k] = ch[k] >= 0 ? ch[k] + wide_off : ~((~ch[k]) + tri_off);
    }
    dst[wide_off + i] = w;
}

}  // namespace
}  // namespace rtsdf

using namespace rtsdf;

struct rtsdf_batch {
    std::vector<rtsdf_ctx*> scenes;
    cudaStream_t stream = nullptr;
    int device = 0;
    // device tables
    SceneDesc* d_desc = nullptr;
    unsigned long long* d_vox_prefix = nullptr;
    unsigned long long* d_tri_prefix = nullptr;
    int2* d_big = nullptr;
    int64_t big_cap = 0;
    WNode* d_wide_all = nullptr;     // all scenes' nodes
    cudaTextureObject_t wtex_all = 0;  // d_wide_all as int4 texels (0: plain loads)
    float4* d_tri_all = nullptr;     // all scenes' leaf triangles
    int64_t wide_cap = 0, tri_cap = 0, total_nt = 0;
    uint32_t* d_ctr = nullptr;   // big_count, bar_count, bar_gen, abort, err
    unsigned long long* d_stamps = nullptr;
    unsigned long long* d_next_ray = nullptr;
    BatchParams* d_params = nullptr;
    BatchParams* h_params = nullptr;   // pinned
    std::vector<SceneDesc> h_desc;
    int max_passes = 0;
    // launch configuration (autotuned)
    int blocks_per_sm = 0;       // 0 = occupancy maximum
    int split_trace = 0;         // trace + finalize as launches of their own after the pipeline launch
    unsigned trace_grid = 0;     // blocks of the split trace launch
    unsigned fin_grid = 0;       // blocks of the split finalize launch
    unsigned long long* d_ray_prefix = nullptr;   // [MAX_BATCH + 1]
    uint32_t* d_jfa_blocks = nullptr;   // split jump flood: [max_passes][ns + 1] block prefix per pass
    size_t jfa_cap = 0;                 // entries of d_jfa_blocks
    std::vector<uint32_t> jfa_total;    // blocks of each pass's launch
    int refill_min = 12;
    int ray_chunk = 1024;
    int leaf_min = 12;
    int use_graph = 1;
    int barrier_spins = 0;
    unsigned grid = 0;
    // CUDA graph of the per-frame pipeline
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = false;
    int64_t frames = 0, launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool own_stream = false;
};

namespace {

rtsdf_status from_cuda_b(cudaError_t e) {
    if (e == cudaSuccess) return RTSDF_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RTSDF_E_OOM;
    }
    return RTSDF_E_CUDA;
}

void drop_graph(rtsdf_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_ok = false;
}

// Rebuild the descriptor table from the scene contexts; returns true when it
// changed (pointers move when a mesh is uploaded or a BVH rebuilt).
cudaError_t refresh_tables(rtsdf_batch* b, bool* changed) {
    const int ns = (int)b->scenes.size();
    std::vector<SceneDesc> desc((size_t)ns);
    std::vector<unsigned long long> vp((size_t)ns + 1), tp((size_t)ns + 1);
    unsigned long long av = 0, at = 0;
    int maxp = 0;
    memset(desc.data(), 0, sizeof(SceneDesc) * desc.size());
    for (int s = 0; s < ns; s++) {
        rtsdf_ctx* c = b->scenes[s];
        SceneDesc& d = desc[s];
        d.t.masked = c->masked;
        d.t.count = c->d_masked_count;
        d.t.nc = c->nc;
        d.t.key0 = (uint32_t)c->cfg.seed;
        d.t.key1 = (uint32_t)(c->cfg.seed >> 32);
        d.t.bx = c->cfg.bmin[0];
        d.t.by = c->cfg.bmin[1];
        d.t.bz = c->cfg.bmin[2];
        d.t.hf = c->hf;
        d.t.wide = c->bvh.wide;
        d.t.tri = c->bvh.tri;
        d.t.nt = c->bvh.nt;
        d.t.coarse = c->coarse;
        d.t.accum = c->accum;
        d.t.counts = c->counts;
        d.t.fine = c->fine;
        d.t.err = c->d_err;
        d.t.ray_min = c->ray_min;
        d.t.ray_cnt = c->ray_cnt;
        d.q = c->qverts;
        d.tris = c->tris;
        d.n_tris = c->nt;
        d.seeds[0] = c->seeds[0];
        d.seeds[1] = c->seeds[1];
        d.hc = c->hc;
        d.beta_vox = c->cfg.beta_vox;
        d.beta_h = c->cfg.beta_vox * c->hc;
        d.alpha = c->cfg.alpha;
        int L = 0;
        while ((1 << L) < c->nc) L++;
        d.passes = L;
        d.nmag = (uint32_t)((0x100000000ull + (unsigned long long)c->nc - 1) / (unsigned long long)c->nc);
        d.t.nc_mag = d.nmag;
        d.t.nearest = c->sign_mode == RTSDF_SIGN_NEAREST;
        maxp = L > maxp ? L : maxp;
        vp[s] = av;
        tp[s] = at;
        av += c->nc3;
        at += (unsigned long long)c->nt;
    }
    vp[ns] = av;
    tp[ns] = at;
    int64_t wo = 0, to = 0;
    for (int s = 0; s < ns; s++) {
        desc[s].wide_off = (int)wo;
        desc[s].tri_off = (int)to;
        wo += b->scenes[s]->bvh.n_wide;
        to += b->scenes[s]->bvh.nt;
    }
    *changed = desc.size() != b->h_desc.size() ||
               memcmp(desc.data(), b->h_desc.data(), sizeof(SceneDesc) * desc.size()) != 0 || maxp != b->max_passes;
    if (!*changed && b->d_desc) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e) return e;
    if (!b->d_desc) {
        if ((e = cudaMalloc(&b->d_desc, sizeof(SceneDesc) * ns))) return e;
        if ((e = cudaMalloc(&b->d_vox_prefix, sizeof(unsigned long long) * (ns + 1)))) return e;
        if ((e = cudaMalloc(&b->d_tri_prefix, sizeof(unsigned long long) * (ns + 1)))) return e;
    }
    if ((int64_t)at > b->big_cap) {
        if (b->d_big) cudaFree(b->d_big);
        b->d_big = nullptr;
        if ((e = cudaMalloc(&b->d_big, sizeof(int2) * (at > 0 ? at : 1)))) return e;
        b->big_cap = (int64_t)at;
    }
    // concatenated BVH of all scenes
    if (wo > b->wide_cap) {
        drop_texture(b->wtex_all);   // the stream is idle (synchronised above)
        if (b->d_wide_all) cudaFree(b->d_wide_all);
        b->d_wide_all = nullptr;
        if ((e = cudaMalloc(&b->d_wide_all, sizeof(WNode) * (wo > 0 ? wo : 1)))) return e;
        b->wide_cap = wo;
        b->wtex_all = make_int4_texture(b->d_wide_all, (sizeof(WNode) / 16) * (size_t)(wo > 0 ? wo : 1), b->device);
    }
    if (to > b->tri_cap) {
        if (b->d_tri_all) cudaFree(b->d_tri_all);
        b->d_tri_all = nullptr;
        if ((e = cudaMalloc(&b->d_tri_all, sizeof(float4) * TRI_F4 * (to > 0 ? to : 1)))) return e;
        b->tri_cap = to;
    }
    b->total_nt = to;
    for (int s = 0; s < ns; s++) {
        const Bvh& bv = b->scenes[s]->bvh;
        if (bv.n_wide > 0) {
            k_rebase_nodes<<<(unsigned)((bv.n_wide + 255) / 256), 256, 0, b->stream>>>(bv.wide, b->d_wide_all,
                                                                                     bv.n_wide, desc[s].wide_off,
                                                                                     desc[s].tri_off);
            b->launches++;
        }
        if (bv.nt > 0 &&
            (e = cudaMemcpyAsync(b->d_tri_all + TRI_F4 * (int64_t)desc[s].tri_off, bv.tri, sizeof(float4) * TRI_F4 * bv.nt,
                                 cudaMemcpyDeviceToDevice, b->stream)))
            return e;
    }
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaStreamSynchronize(b->stream))) return e;
    if ((e = cudaMemcpy(b->d_desc, desc.data(), sizeof(SceneDesc) * ns, cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(b->d_vox_prefix, vp.data(), sizeof(unsigned long long) * (ns + 1), cudaMemcpyHostToDevice)))
        return e;
    if ((e = cudaMemcpy(b->d_tri_prefix, tp.data(), sizeof(unsigned long long) * (ns + 1), cudaMemcpyHostToDevice)))
        return e;
    // split jump flood: per pass, the z-blocked pass's blocks of every
    // scene that has the pass (32 x 4 columns of T = 8 lattice voxels)
    {
        const size_t rows = (size_t)maxp, cols = (size_t)ns + 1;
        std::vector<uint32_t> pre(rows * cols, 0u);
        b->jfa_total.assign(rows, 0u);
        for (int p = 0; p < maxp; p++) {
            uint64_t acc = 0;
            for (int s = 0; s < ns; s++) {
                pre[(size_t)p * cols + s] = (uint32_t)acc;
                const int L = desc[s].passes, n = desc[s].t.nc;
                if (p < L) {
                    const uint64_t k = 1ull << (L - 1 - p), lat = ((uint64_t)n + k - 1) / k;
                    acc += (uint64_t)((n + 31) / 32) * (uint64_t)((n + 3) / 4) * ((lat + 7) / 8) * k;
                }
            }
            if (acc > 0x7FFFFFFFull) return cudaErrorInvalidValue;
            pre[(size_t)p * cols + ns] = (uint32_t)acc;
            b->jfa_total[p] = (uint32_t)acc;
        }
        if (rows * cols > b->jfa_cap) {
            if (b->d_jfa_blocks) cudaFree(b->d_jfa_blocks);
            b->d_jfa_blocks = nullptr;
            b->jfa_cap = 0;
            if ((e = cudaMalloc(&b->d_jfa_blocks, sizeof(uint32_t) * rows * cols))) return e;
            b->jfa_cap = rows * cols;
        }
        if (rows > 0 &&
            (e = cudaMemcpy(b->d_jfa_blocks, pre.data(), sizeof(uint32_t) * rows * cols, cudaMemcpyHostToDevice)))
            return e;
    }
    b->h_desc = desc;
    b->max_passes = maxp;
    *changed = true;
    return cudaSuccess;
}

cudaError_t launch_frame_kernel(rtsdf_batch* b) {
    BatchArgs a;
    a.sc = b->d_desc;
    a.ns = (int)b->scenes.size();
    a.params = b->d_params;
    a.vox_prefix = b->d_vox_prefix;
    a.tri_prefix = b->d_tri_prefix;
    a.max_passes = b->max_passes;
    a.big_list = b->d_big;
    a.big_count = b->d_ctr + 0;
    a.bar_count = b->d_ctr + 1;
    a.bar_gen = b->d_ctr + 2;
    a.abort = b->d_ctr + 3;
    a.err = b->d_ctr + 4;
    a.next_ray = b->d_next_ray;
    a.refill_min = b->refill_min;
    a.ray_chunk = b->ray_chunk;
    a.leaf_min = b->leaf_min;
    a.spins = b->barrier_spins > 0 ? (uint32_t)b->barrier_spins : BARRIER_SPINS;
    a.stamps = b->d_stamps;
    a.bvh.wide = b->d_wide_all;
    a.bvh.wtex = texture_fetch_on() ? b->wtex_all : 0;
    a.bvh.tri = b->d_tri_all;
    a.bvh.nt = b->total_nt;
    a.bvh.err = b->d_ctr + 4;
    a.split = b->split_trace;
    a.ray_prefix = b->d_ray_prefix;
    a.fin_done = b->d_ctr + 5;
    a.jfa_blocks = b->d_jfa_blocks;
    a.phase = b->split_trace ? 1 : 0;
    void* args[] = {&a};
    b->launches++;
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_batch_frame, dim3(b->grid), dim3(TRACE_THREADS), args,
                                                0, b->stream);
    if (e || !b->split_trace) return e;
    // split form: the jump flood as one launch per pass, the rest of the
    // pipeline (mask, ray prefix) as a second cooperative launch, then the
    // trace and the finalize
    for (int p = 0; p < b->max_passes; p++) {
        if (b->jfa_total[p] == 0) continue;
        k_batch_jfa<<<b->jfa_total[p], dim3(32, 4, 1), 0, b->stream>>>(a, p);
        b->launches++;
    }
    a.phase = 2;
    b->launches++;
    e = cudaLaunchCooperativeKernel((const void*)k_batch_frame, dim3(b->grid), dim3(TRACE_THREADS), args, 0,
                                    b->stream);
    if (e) return e;
    b->launches += 2;
    if (a.bvh.wtex) k_batch_trace<true><<<b->trace_grid, TRACE_THREADS, 0, b->stream>>>(a);
    else k_batch_trace<false><<<b->trace_grid, TRACE_THREADS, 0, b->stream>>>(a);
    k_batch_finalize<<<b->fin_grid, 256, 0, b->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t ensure_grid(rtsdf_batch* b) {
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_frame, TRACE_THREADS, 0);
    if (e) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int use = (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) ? b->blocks_per_sm : per_sm;
    const unsigned g = (unsigned)(sms * use);
    int tper = 0;
    if (b->wtex_all && texture_fetch_on())
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tper, k_batch_trace<true>, TRACE_THREADS, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tper, k_batch_trace<false>, TRACE_THREADS, 0);
    if (e) return e;
    if (tper < 1) return cudaErrorInvalidConfiguration;
    const unsigned tg = (unsigned)(sms * tper), fg = (unsigned)(sms * 8);
    if (g != b->grid || tg != b->trace_grid || fg != b->fin_grid) {
        b->grid = g;
        b->trace_grid = tg;
        b->fin_grid = fg;
        drop_graph(b);
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

rtsdf_status rtsdf_batch_create(const rtsdf_config* cfgs, int32_t n, rtsdf_batch_t* out) {
    if (!cfgs || !out || n < 1 || n > MAX_BATCH) return RTSDF_E_ARG;
    *out = nullptr;
    rtsdf_batch* b = new (std::nothrow) rtsdf_batch();
    if (!b) return RTSDF_E_OOM;
    cudaGetDevice(&b->device);
    // graph capture needs a stream other than the legacy default stream
    b->stream = (cudaStream_t)cfgs[0].stream;
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return RTSDF_E_CUDA;
        }
        b->own_stream = true;
    }
    rtsdf_status st = RTSDF_OK;
    for (int i = 0; i < n && st == RTSDF_OK; i++) {
        rtsdf_config c = cfgs[i];
        c.stream = b->stream;
        rtsdf_t ctx = nullptr;
        st = rtsdf_create(&c, &ctx);
        if (st == RTSDF_OK) b->scenes.push_back(ctx);
    }
    cudaError_t e = cudaSuccess;
    if (st == RTSDF_OK) {
        if (!e) e = cudaMalloc(&b->d_ctr, sizeof(uint32_t) * 8);
        if (!e) e = cudaMemset(b->d_ctr, 0, sizeof(uint32_t) * 8);
        if (!e) e = cudaMalloc(&b->d_next_ray, sizeof(unsigned long long));
        if (!e) e = cudaMalloc(&b->d_ray_prefix, sizeof(unsigned long long) * (MAX_BATCH + 1));
        if (!e) e = cudaMalloc(&b->d_stamps, sizeof(unsigned long long) * 8);
        if (!e) e = cudaMemset(b->d_stamps, 0, sizeof(unsigned long long) * 8);
        if (!e) e = cudaMalloc(&b->d_params, sizeof(BatchParams));
        if (!e) e = cudaMallocHost(&b->h_params, sizeof(BatchParams));
        if (!e) e = cudaEventCreate(&b->ev0);
        if (!e) e = cudaEventCreate(&b->ev1);
        if (e) st = from_cuda_b(e);
    }
    if (st != RTSDF_OK) {
        rtsdf_batch_destroy(b);
        return st;
    }
    *out = b;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_destroy(rtsdf_batch_t b) {
    if (!b) return RTSDF_E_ARG;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (rtsdf_ctx* c : b->scenes) rtsdf_destroy(c);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_vox_prefix) cudaFree(b->d_vox_prefix);
    if (b->d_tri_prefix) cudaFree(b->d_tri_prefix);
    if (b->d_big) cudaFree(b->d_big);
    drop_texture(b->wtex_all);
    if (b->d_wide_all) cudaFree(b->d_wide_all);
    if (b->d_tri_all) cudaFree(b->d_tri_all);
    if (b->d_ctr) cudaFree(b->d_ctr);
    if (b->d_next_ray) cudaFree(b->d_next_ray);
    if (b->d_stamps) cudaFree(b->d_stamps);
    if (b->d_ray_prefix) cudaFree(b->d_ray_prefix);
    if (b->d_jfa_blocks) cudaFree(b->d_jfa_blocks);
    if (b->d_params) cudaFree(b->d_params);
    if (b->h_params) cudaFreeHost(b->h_params);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_context(rtsdf_batch_t b, int32_t i, rtsdf_t* out) {
    if (!b || !out || i < 0 || i >= (int32_t)b->scenes.size()) return RTSDF_E_ARG;
    *out = b->scenes[(size_t)i];
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_set_tuning(rtsdf_batch_t b, const rtsdf_batch_tuning* t) {
    if (!b || !t) return RTSDF_E_ARG;
    if (t->blocks_per_sm < 0 || t->refill_min < 1 || t->refill_min > 32 || t->ray_chunk < 32 ||
        t->ray_chunk > (1 << 20))
        return RTSDF_E_ARG;
    if (t->barrier_spins < 0 || t->leaf_min < 1 || t->leaf_min > 32) return RTSDF_E_ARG;
    if (t->split_trace != 0 && t->split_trace != 1) return RTSDF_E_ARG;
    if (t->blocks_per_sm != b->blocks_per_sm || t->refill_min != b->refill_min || t->ray_chunk != b->ray_chunk ||
        t->use_graph != b->use_graph || t->barrier_spins != b->barrier_spins || t->leaf_min != b->leaf_min ||
        t->split_trace != b->split_trace)
        drop_graph(b);
    b->split_trace = t->split_trace;
    b->leaf_min = t->leaf_min;
    b->barrier_spins = t->barrier_spins;
    b->blocks_per_sm = t->blocks_per_sm;
    b->refill_min = t->refill_min;
    b->ray_chunk = t->ray_chunk;
    b->use_graph = t->use_graph;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_get_tuning(rtsdf_batch_t b, rtsdf_batch_tuning* t) {
    if (!b || !t) return RTSDF_E_ARG;
    t->blocks_per_sm = b->blocks_per_sm;
    t->refill_min = b->refill_min;
    t->ray_chunk = b->ray_chunk;
    t->use_graph = b->use_graph;
    t->barrier_spins = b->barrier_spins;
    t->leaf_min = b->leaf_min;
    t->split_trace = b->split_trace;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_frame(rtsdf_batch_t b, float d_vox, int32_t rays, int32_t frame) {
    if (!b) return RTSDF_E_ARG;
    if (!isfinite(d_vox) || rays < 1 || rays > 1024 || (rays & (rays - 1)) || frame < 0) return RTSDF_E_ARG;
    for (rtsdf_ctx* c : b->scenes)
        if (!c->have_mesh || !c->bvh.built || c->bvh_dirty || c->reset_pending) return RTSDF_E_STATE;
    bool changed = false;
    cudaError_t e = refresh_tables(b, &changed);
    if (!e) e = ensure_grid(b);
    if (e) return from_cuda_b(e);
    if (changed) drop_graph(b);
    // the per-frame parameters travel through a pinned host block that the
    // graph copies to the device at its start, so one graph serves all frames
    e = cudaStreamSynchronize(b->stream);   // the previous frame's copy has consumed h_params
    if (e) return from_cuda_b(e);
    int lg = 0;
    while ((1 << lg) < rays) lg++;
    b->h_params->frame = (uint32_t)frame;
    b->h_params->rays = rays;
    b->h_params->log2_rays = lg;
    b->h_params->d_vox = d_vox;
    if (b->use_graph && !b->graph_ok && !b->exec) {
        // capture once: parameter copy + the persistent kernel
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            // barrier words (count, generation, abort) start at zero every frame
            cudaError_t e1 = cudaMemsetAsync(b->d_ctr + 1, 0, 3 * sizeof(uint32_t), b->stream);
            if (!e1) e1 = cudaMemsetAsync(b->d_ctr + 5, 0, sizeof(uint32_t), b->stream);
            if (!e1)
                e1 = cudaMemcpyAsync(b->d_params, b->h_params, sizeof(BatchParams), cudaMemcpyHostToDevice, b->stream);
            cudaError_t e2 = e1 ? e1 : launch_frame_kernel(b);
            b->launches--;   // counted at replay
            cudaGraph_t g = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
            if (!e2 && !e3 && g) {
                if (cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
                    b->graph = g;
                    b->graph_ok = true;
                } else {
                    cudaGraphDestroy(g);
                }
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();   // a capture that the driver refused leaves no sticky error
        if (!b->graph_ok) b->use_graph = 0;   // fall back to direct launches
    }
    cudaEventRecord(b->ev0, b->stream);
    if (b->graph_ok) {
        e = cudaGraphLaunch(b->exec, b->stream);
        b->launches++;
    } else {
        e = cudaMemsetAsync(b->d_ctr + 1, 0, 3 * sizeof(uint32_t), b->stream);
        if (!e) e = cudaMemsetAsync(b->d_ctr + 5, 0, sizeof(uint32_t), b->stream);
        if (!e) e = cudaMemcpyAsync(b->d_params, b->h_params, sizeof(BatchParams), cudaMemcpyHostToDevice, b->stream);
        if (!e) e = launch_frame_kernel(b);
    }
    cudaEventRecord(b->ev1, b->stream);
    if (e) return from_cuda_b(e);
    for (rtsdf_ctx* c : b->scenes) {
        int L = 0;
        while ((1 << L) < c->nc) L++;
        c->cur = L & 1;
        c->jfa_passes = L;
        c->voxelized = c->flooded = true;
    }
    b->frames++;
    return RTSDF_OK;
}

rtsdf_status rtsdf_batch_sync(rtsdf_batch_t b) {
    if (!b) return RTSDF_E_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e) return from_cuda_b(e);
    uint32_t ctr[5];
    if ((e = cudaMemcpy(ctr, b->d_ctr, sizeof(ctr), cudaMemcpyDeviceToHost))) return from_cuda_b(e);
    if (ctr[4]) {   // the error word is read once
        if ((e = cudaMemset(b->d_ctr + 4, 0, sizeof(uint32_t)))) return from_cuda_b(e);
    }
    rtsdf_status worst = RTSDF_OK;
    if (ctr[4] & ERR_TIMEOUT) worst = RTSDF_E_TIMEOUT;
    for (rtsdf_ctx* c : b->scenes) {
        rtsdf_status s = rtsdf_sync(c);
        if (s != RTSDF_OK && worst == RTSDF_OK) worst = s;
    }
    return worst;
}

rtsdf_status rtsdf_batch_stats(rtsdf_batch_t b, rtsdf_batch_info* out) {
    if (!b || !out) return RTSDF_E_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e) return from_cuda_b(e);
    memset(out, 0, sizeof(*out));
    out->n_scenes = (int32_t)b->scenes.size();
    out->grid = (int32_t)b->grid;
    out->graph = b->graph_ok ? 1 : 0;
    out->frames = b->frames;
    out->launches = b->launches;
    float ms = -1.f;
    if (b->frames > 0 && cudaEventElapsedTime(&ms, b->ev0, b->ev1) != cudaSuccess) ms = -1.f;
    out->last_frame_ms = ms;
    unsigned long long st[8];
    if (cudaMemcpy(st, b->d_stamps, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess)
        for (int k = 0; k < 7; k++) out->stage_ms[k] = st[k + 1] >= st[k] ? (float)((st[k + 1] - st[k]) * 1e-6) : 0.f;
    return RTSDF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner of the batched form (see rtsdf_batch_autotune in rtsdf.h).
namespace {

std::mutex g_bt_mutex;
std::map<std::string, rtsdf_batch_tuning> g_bt_cache;

struct BatchSnapshot {
    std::vector<void*> bufs;
    cudaError_t take(rtsdf_batch* b) {
        for (rtsdf_ctx* c : b->scenes) {
            const size_t bytes = c->nf3 * 4;
            for (int k = 0; k < 3; k++) {
                void* p = nullptr;
                cudaError_t e = cudaMalloc(&p, bytes);
                if (e) return e;
                bufs.push_back(p);
                const void* src = k == 0 ? (const void*)c->accum : k == 1 ? (const void*)c->counts : (const void*)c->fine;
                if ((e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToDevice, b->stream))) return e;
            }
        }
        return cudaSuccess;
    }
    cudaError_t restore(rtsdf_batch* b) const {
        size_t i = 0;
        for (rtsdf_ctx* c : b->scenes) {
            const size_t bytes = c->nf3 * 4;
            void* dst[3] = {c->accum, c->counts, c->fine};
            for (int k = 0; k < 3; k++) {
                cudaError_t e = cudaMemcpyAsync(dst[k], bufs[i++], bytes, cudaMemcpyDeviceToDevice, b->stream);
                if (e) return e;
            }
        }
        return cudaSuccess;
    }
    ~BatchSnapshot() {
        for (void* p : bufs) cudaFree(p);
    }
};

}  // namespace

extern "C" rtsdf_status rtsdf_batch_autotune(rtsdf_batch_t b, float d_vox, int32_t rays, int32_t frame,
                                             int32_t use_cache, rtsdf_batch_tuning* best) {
    if (!b) return RTSDF_E_ARG;
    unsigned long long vox = 0, tris = 0;
    for (rtsdf_ctx* c : b->scenes) {
        vox += c->nc3;
        tris += (unsigned long long)c->nt;
    }
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, b->device);
    int lv = 0, lt = 0;
    while ((1ull << lv) < vox) lv++;
    while ((1ull << lt) < tris) lt++;
    char kbuf[320];
    snprintf(kbuf, sizeof(kbuf), "%s|%zu|%d|%d", prop.name, b->scenes.size(), lv, lt);
    const std::string key = kbuf;
    rtsdf_batch_tuning cur;
    rtsdf_batch_get_tuning(b, &cur);
    if (use_cache) {
        std::lock_guard<std::mutex> lock(g_bt_mutex);
        auto it = g_bt_cache.find(key);
        if (it != g_bt_cache.end()) {
            rtsdf_status s = rtsdf_batch_set_tuning(b, &it->second);
            if (s == RTSDF_OK && best) *best = it->second;
            return s;
        }
    }
    BatchSnapshot snap;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (!e) e = snap.take(b);
    if (e) return from_cuda_b(e);
    // one timed frame per candidate from the saved state (the events bracket
    // only the replay, not the graph capture)
    auto trial = [&](const rtsdf_batch_tuning& t, float* ms) -> rtsdf_status {
        rtsdf_status s = rtsdf_batch_set_tuning(b, &t);
        if (s == RTSDF_OK) {
            cudaError_t r = snap.restore(b);
            if (r) return from_cuda_b(r);
            s = rtsdf_batch_frame(b, d_vox, rays, frame);
            if (s == RTSDF_OK) s = rtsdf_batch_sync(b);
        }
        if (s != RTSDF_OK) return s;
        float v = 0.f;
        if (cudaEventElapsedTime(&v, b->ev0, b->ev1) != cudaSuccess) return RTSDF_E_CUDA;
        *ms = v;
        return RTSDF_OK;
    };
    float base = 0.f;
    rtsdf_status st = trial(cur, &base);
    // one persistent launch for every stage, or the trace and finalize as
    // launches of their own (at the tracer's own occupancy)
    if (st == RTSDF_OK) {
        rtsdf_batch_tuning t = cur;
        t.split_trace = 1 - cur.split_trace;
        float ms = 0.f;
        st = trial(t, &ms);
        if (st == RTSDF_OK && ms < base) {
            base = ms;
            cur = t;
        }
    }
    const int refills[] = {4, 8, 12, 16, 20};
    for (int r : refills) {
        if (st != RTSDF_OK || r == cur.refill_min) continue;
        rtsdf_batch_tuning t = cur;
        t.refill_min = r;
        float ms = 0.f;
        st = trial(t, &ms);
        if (st == RTSDF_OK && ms < base) {
            base = ms;
            cur = t;
        }
    }
    const int leafs[] = {8, 12, 16, 24};
    for (int lm : leafs) {
        if (st != RTSDF_OK || lm == cur.leaf_min) continue;
        rtsdf_batch_tuning t = cur;
        t.leaf_min = lm;
        float ms = 0.f;
        st = trial(t, &ms);
        if (st == RTSDF_OK && ms < base) {
            base = ms;
            cur = t;
        }
    }
    const int chunks[] = {64, 256, 1024};
    for (int ch : chunks) {
        if (st != RTSDF_OK || ch == cur.ray_chunk) continue;
        rtsdf_batch_tuning t = cur;
        t.ray_chunk = ch;
        float ms = 0.f;
        st = trial(t, &ms);
        if (st == RTSDF_OK && ms < base) {
            base = ms;
            cur = t;
        }
    }
    int per_sm = 0;
    if (st == RTSDF_OK &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_frame, TRACE_THREADS, 0) != cudaSuccess)
        st = RTSDF_E_CUDA;
    for (int blocks = per_sm - 1; blocks >= per_sm - 2 && blocks >= 1 && st == RTSDF_OK; blocks--) {
        rtsdf_batch_tuning t = cur;
        t.blocks_per_sm = blocks;
        float ms = 0.f;
        st = trial(t, &ms);
        if (st == RTSDF_OK && ms < base) {
            base = ms;
            cur = t;
        }
    }
    rtsdf_status s2 = rtsdf_batch_set_tuning(b, &cur);
    cudaError_t r = snap.restore(b);
    if (!r) r = cudaStreamSynchronize(b->stream);
    if (st != RTSDF_OK) return st;
    if (s2 != RTSDF_OK) return s2;
    if (r) return from_cuda_b(r);
    {
        std::lock_guard<std::mutex> lock(g_bt_mutex);
        g_bt_cache[key] = cur;
    }
    if (best) *best = cur;
    return RTSDF_OK;
}
