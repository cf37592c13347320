// Launch-parameter tuning of the per-scene path: rtsdf_set_tuning /
// rtsdf_get_tuning and the autotuner rtsdf_autotune.
//
// The autotuner times candidates with CUDA events on the caller's own scene:
// the jump-flood tile on rtsdf_jfa (re-voxelizing before each candidate so
// every run starts from the same seeds), then the tracer's refill threshold,
// ray chunk and persistent blocks per SM by coordinate descent on the mask +
// trace of one frame.  The temporal state (accumulator, counts, fine SDF) is
// copied aside first and restored before every tracer candidate and at the
// end, so tuning does not change the accumulated SDF.  Winners are cached
// per (device, coarse_n, log2 triangles).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.cuh"

using namespace rtsdf;

namespace {

std::mutex g_mutex;
std::map<std::string, rtsdf_tuning> g_cache;

rtsdf_status from_cuda_t(cudaError_t e) {
    if (e == cudaSuccess) return RTSDF_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RTSDF_E_OOM;
    }
    return RTSDF_E_CUDA;
}

bool valid(const rtsdf_tuning& t) {
    return t.jfa_tile >= 0 && t.jfa_tile <= 4 && t.trace_blocks_per_sm >= 0 && t.refill_min >= 1 &&
           t.refill_min <= 32 && t.ray_chunk >= 32 && t.ray_chunk <= (1 << 20) && t.leaf_min >= 1 &&
           t.leaf_min <= 32;
}

std::string cache_key(rtsdf_ctx* c) {
    cudaDeviceProp p;
    memset(&p, 0, sizeof(p));
    cudaGetDeviceProperties(&p, c->device);
    int lt = 0;
    while ((1ll << lt) < c->nt) lt++;
    char buf[320];
    snprintf(buf, sizeof(buf), "%s|%d|%d", p.name, c->nc, lt);
    return buf;
}

struct Snapshot {
    float* accum = nullptr;
    uint32_t* counts = nullptr;
    float* fine = nullptr;
    cudaError_t take(rtsdf_ctx* c) {
        cudaError_t e = cudaMalloc(&accum, c->nf3 * sizeof(float));
        if (!e) e = cudaMalloc(&counts, c->nf3 * sizeof(uint32_t));
        if (!e) e = cudaMalloc(&fine, c->nf3 * sizeof(float));
        if (!e) e = cudaMemcpyAsync(accum, c->accum, c->nf3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        if (!e) e = cudaMemcpyAsync(counts, c->counts, c->nf3 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream);
        if (!e) e = cudaMemcpyAsync(fine, c->fine, c->nf3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        return e;
    }
    cudaError_t restore(rtsdf_ctx* c) const {
        cudaError_t e = cudaMemcpyAsync(c->accum, accum, c->nf3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        if (!e) e = cudaMemcpyAsync(c->counts, counts, c->nf3 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream);
        if (!e) e = cudaMemcpyAsync(c->fine, fine, c->nf3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        return e;
    }
    ~Snapshot() {
        if (accum) cudaFree(accum);
        if (counts) cudaFree(counts);
        if (fine) cudaFree(fine);
    }
};

// device time of fn() on the context's stream, best of `reps`
template <class F>
cudaError_t time_ms(rtsdf_ctx* c, cudaEvent_t a, cudaEvent_t b, int reps, F fn, float* out) {
    float best = 1e30f;
    for (int i = 0; i < reps; i++) {
        cudaError_t e = cudaEventRecord(a, c->stream);
        if (!e) e = fn();
        if (!e) e = cudaEventRecord(b, c->stream);
        if (!e) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, a, b);
        if (e) return e;
        best = ms < best ? ms : best;
    }
    *out = best;
    return cudaSuccess;
}

}  // namespace

extern "C" {

rtsdf_status rtsdf_set_tuning(rtsdf_t c, const rtsdf_tuning* t) {
    if (!c || !t || !valid(*t)) return RTSDF_E_ARG;
    c->tune = *t;
    return RTSDF_OK;
}

rtsdf_status rtsdf_get_tuning(rtsdf_t c, rtsdf_tuning* t) {
    if (!c || !t) return RTSDF_E_ARG;
    *t = c->tune;
    return RTSDF_OK;
}

rtsdf_status rtsdf_autotune(rtsdf_t c, float d_vox, int32_t rays, int32_t frame, int32_t use_cache,
                            rtsdf_tuning* best) {
    if (!c) return RTSDF_E_ARG;
    if (!isfinite(d_vox) || rays < 1 || rays > 1024 || (rays & (rays - 1)) || frame < 0) return RTSDF_E_ARG;
    if (!c->have_mesh || !c->bvh.built || c->bvh_dirty) return RTSDF_E_STATE;
    const std::string key = cache_key(c);
    if (use_cache) {
        std::lock_guard<std::mutex> lock(g_mutex);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            c->tune = it->second;
            if (best) *best = it->second;
            return RTSDF_OK;
        }
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    Snapshot snap;
    if (!e) e = snap.take(c);
    const bool reset0 = c->reset_pending;
    rtsdf_tuning cur = c->tune;
    // jump-flood tile
    float best_ms = 1e30f;
    for (int tile = 0; tile < 5 && !e; tile++) {
        c->tune = cur;
        c->tune.jfa_tile = tile;
        float ms = 0.f;
        e = time_ms(c, a, b, 2, [&]() {
            cudaError_t r = launch_voxelize(c);
            return r ? r : launch_jfa(c);
        }, &ms);
        if (!e && ms < best_ms) {
            best_ms = ms;
            cur.jfa_tile = tile;
        }
    }
    c->tune = cur;
    if (!e) e = launch_voxelize(c);
    if (!e) e = launch_jfa(c);
    // tracer knobs, one coordinate at a time
    auto trial = [&](const rtsdf_tuning& t, float* ms) {
        c->tune = t;
        cudaError_t r = snap.restore(c);
        if (r) return r;
        c->reset_pending = reset0;
        return time_ms(c, a, b, 1, [&]() {
            cudaError_t q = launch_mask(c, d_vox);
            return q ? q : launch_trace(c, rays, frame);
        }, ms);
    };
    float base = 0.f;
    if (!e) e = trial(cur, &base);
    const int refills[] = {4, 8, 12, 16, 20};
    for (int r : refills) {
        if (e || r == cur.refill_min) continue;
        rtsdf_tuning t = cur;
        t.refill_min = r;
        float ms = 0.f;
        e = trial(t, &ms);
        if (!e && ms < base) {
            base = ms;
            cur = t;
        }
    }
    const int leafs[] = {8, 12, 16, 24};
    for (int lm : leafs) {
        if (e || lm == cur.leaf_min) continue;
        rtsdf_tuning t = cur;
        t.leaf_min = lm;
        float ms = 0.f;
        e = trial(t, &ms);
        if (!e && ms < base) {
            base = ms;
            cur = t;
        }
    }
    const int chunks[] = {64, 256, 1024};
    for (int ch : chunks) {
        if (e || ch == cur.ray_chunk) continue;
        rtsdf_tuning t = cur;
        t.ray_chunk = ch;
        float ms = 0.f;
        e = trial(t, &ms);
        if (!e && ms < base) {
            base = ms;
            cur = t;
        }
    }
    int per_sm = 0;
    if (!e) e = trace_occupancy(&per_sm);
    for (int blocks = per_sm - 1; blocks >= per_sm - 2 && blocks >= 1 && !e; blocks--) {
        rtsdf_tuning t = cur;
        t.trace_blocks_per_sm = blocks;
        float ms = 0.f;
        e = trial(t, &ms);
        if (!e && ms < base) {
            base = ms;
            cur = t;
        }
    }
    c->tune = cur;
    if (!e) e = snap.restore(c);
    c->reset_pending = reset0;
    c->voxelized = c->flooded = true;
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e) return from_cuda_t(e);
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        g_cache[key] = cur;
    }
    if (best) *best = cur;
    return RTSDF_OK;
}

}  // extern "C"
