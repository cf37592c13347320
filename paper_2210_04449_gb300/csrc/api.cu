// extern "C" entry points of librtsdf: argument checks, the call-order state
// machine, device memory ownership, the device status word and per-stage
// timing.  The numerical work is in the stage translation units.
#include <atomic>
#include <math.h>
#include <math_constants.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <nvtx3/nvToolsExt.h>
#include <vector>

#include "internal.cuh"

using namespace rtsdf;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

rtsdf_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RTSDF_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RTSDF_E_OOM;
    }
    return RTSDF_E_CUDA;
}

__global__ void k_fill_f32(float* p, size_t n, float v) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

cudaError_t fill_f32(rtsdf_ctx* c, float* p, size_t n, float v) {
    if (n == 0) return cudaSuccess;
    RTSDF_LAUNCH(c, k_fill_f32, (unsigned)((n + 255) / 256), 256, 0, p, n, v);
    return cudaGetLastError();
}

__global__ void k_check_objects(const int32_t* vobj, int64_t nv, int n_obj, uint32_t* err, int32_t* fixed) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    int o = vobj[i];
    if (o < 0 || o >= n_obj) {
        atomicOr(err, ERR_MESH);
        o = 0;
    }
    fixed[i] = o;
}

// Allocation-failure injection for tests (rtsdf_debug_fail_allocation):
// the number of device allocations that still succeed before one fails,
// -1 when off.
std::atomic<long long> g_fail_after{-1};

// Texture-path switch for tests (rtsdf_debug_texture_fetch), on by default.
std::atomic<bool> g_texture_fetch{true};

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    long long k = g_fail_after.load();
    while (k >= 0) {
        if (g_fail_after.compare_exchange_weak(k, k - 1)) {
            if (k == 0) return cudaErrorMemoryAllocation;   // the injected failure (the hook is now off)
            break;
        }
    }
    return cudaMalloc((void**)p, count > 0 ? count * sizeof(T) : 16);
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_all(rtsdf_ctx* c) {
    dfree(c->verts); dfree(c->qverts); dfree(c->tris); dfree(c->vert_obj); dfree(c->obj_box);
    dfree(c->obj_trans); dfree(c->obj_xform); dfree(c->moved_list); dfree(c->d_moved_count);
    dfree(c->seeds[0]); dfree(c->seeds[1]); dfree(c->coarse); dfree(c->big_list); dfree(c->d_big_count);
    dfree(c->accum); dfree(c->counts); dfree(c->fine); dfree(c->masked); dfree(c->d_masked_count);
    dfree(c->ray_min); dfree(c->ray_cnt); dfree(c->d_next_ray);
    dfree(c->bin_count); dfree(c->bin_start); dfree(c->bin_cursor); dfree(c->bin_items); dfree(c->bin_overflow);
    drop_texture(c->bvh.wtex);
    dfree(c->bvh.nodes); dfree(c->bvh.wide); dfree(c->bvh.nbox); dfree(c->bvh.lbox); dfree(c->bvh.tri); dfree(c->bvh.leaf_tri); dfree(c->bvh.leaf_parent); dfree(c->bvh.flags);
    dfree(c->bvh.col_fb); dfree(c->bvh.col_fslot); dfree(c->bvh.col_nb); dfree(c->bvh.col_nslot);
    dfree(c->bvh.col_kids); dfree(c->bvh.col_nint); dfree(c->bvh.col_total);
    dfree(c->bvh.root); dfree(c->bvh.mk0); dfree(c->bvh.mk1); dfree(c->bvh.mv0); dfree(c->bvh.mv1);
    dfree(c->bvh.hist); dfree(c->bvh.d_depth); dfree(c->bvh.sah);
    dfree(c->bvh.top_child); dfree(c->bvh.top_ids); dfree(c->bvh.top_box); dfree(c->bvh.top_scratch);
    dfree(c->bvh.obj_count);
    dfree(c->d_err);
    dfree(c->d_counters);
    for (auto& t : c->timers) {
        for (int i = 0; i < TIMER_RING; i++) {
            if (t.a[i]) cudaEventDestroy(t.a[i]);
            if (t.b[i]) cudaEventDestroy(t.b[i]);
            t.a[i] = t.b[i] = nullptr;
        }
        t.n = 0;
    }
}

cudaError_t reset_temporal(rtsdf_ctx* c) {
    cudaError_t e = fill_f32(c, c->accum, c->nf3, INFINITY);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->counts, 0, c->nf3 * sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fine, 0, c->nf3 * sizeof(float), c->stream);
    return e;
}

// Per-slot frame scratch back to "nothing committed" for the context's sign
// mode (after a mode change).
cudaError_t reset_scratch(rtsdf_ctx* c) {
    const bool nearest = c->sign_mode == RTSDF_SIGN_NEAREST;
    cudaError_t e = nearest ? cudaMemsetAsync(c->ray_min, 0xFF, 8 * c->nc3 * sizeof(uint32_t), c->stream)
                            : fill_f32(c, reinterpret_cast<float*>(c->ray_min), 8 * c->nc3, INFINITY);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ray_cnt, 0, 8 * c->nc3 * sizeof(uint32_t), c->stream);
    return e;
}

// sum the recorded event pairs of one stage into its carry (waits for them)
void drain(Timer& t) {
    for (int i = 0; i < t.n; i++) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b[i]) == cudaSuccess && cudaEventElapsedTime(&ms, t.a[i], t.b[i]) == cudaSuccess) {
            t.carry_ms += ms;
            t.carry_calls++;
        }
    }
    t.n = 0;
}

// Each stage call is also an NVTX range (named for profilers such as ncu's
// range filters; the header-only NVTX v3 API costs a pointer test when no
// tool is attached).
const char* const kStageRange[ST_COUNT] = {"rtsdf voxelize", "rtsdf jfa", "rtsdf mask",   "rtsdf trace",
                                           "rtsdf bvh",      "rtsdf shadow", "rtsdf shadow backward",
                                           "rtsdf motion"};

struct StageTimer {
    rtsdf_ctx* c;
    Stage s;
    int slot = -1;
    StageTimer(rtsdf_ctx* ctx, Stage st) : c(ctx), s(st) {
        nvtxRangePushA(kStageRange[s]);
        if (!c->profiling) return;
        Timer& t = c->timers[s];
        if (t.n == TIMER_RING) drain(t);
        slot = t.n;
        cudaEventRecord(t.a[slot], c->stream);
    }
    ~StageTimer() {
        nvtxRangePop();
        if (slot < 0) return;
        Timer& t = c->timers[s];
        cudaEventRecord(t.b[slot], c->stream);
        t.n = slot + 1;
    }
};

// read (and clear) the device status word; synchronises the stream
rtsdf_status sync_status(rtsdf_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    uint32_t err = 0;
    e = cudaMemcpy(&err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    if (err) {
        e = cudaMemset(c->d_err, 0, sizeof(uint32_t));
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (err & ERR_MESH) return RTSDF_E_MESH;
    if (err & ERR_STACK) return RTSDF_E_OVERFLOW;
    if (err & ERR_TIMEOUT) return RTSDF_E_TIMEOUT;
    return RTSDF_OK;
}

bool finite3(const float v[3]) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

}  // namespace

bool rtsdf::texture_fetch_on() { return g_texture_fetch.load(); }

extern "C" {

rtsdf_status rtsdf_create(const rtsdf_config* cfg, rtsdf_t* out) {
    if (!cfg || !out) return RTSDF_E_ARG;
    *out = nullptr;
    if (!(cfg->extent > 0.f) || !isfinite(cfg->extent) || !finite3(cfg->bmin)) return RTSDF_E_ARG;
    if (cfg->coarse_n < 1 || cfg->coarse_n > MAX_N) return RTSDF_E_ARG;
    if (!(cfg->beta_vox >= 0.f) || !isfinite(cfg->beta_vox)) return RTSDF_E_ARG;
    if (!(cfg->alpha >= 0.f && cfg->alpha <= 1.f)) return RTSDF_E_ARG;
    rtsdf_ctx* c = new (std::nothrow) rtsdf_ctx();
    if (!c) return RTSDF_E_OOM;
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cfg->stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return RTSDF_E_CUDA;
    }
    c->nc = cfg->coarse_n;
    c->nf = 2 * cfg->coarse_n;
    c->nc3 = (size_t)c->nc * c->nc * c->nc;
    c->nf3 = (size_t)c->nf * c->nf * c->nf;
    c->hc = cfg->extent / (float)c->nc;
    c->hf = cfg->extent / (float)c->nf;
    cudaError_t e = cudaSuccess;
    if (!e) e = dalloc(&c->seeds[0], c->nc3);
    if (!e) e = dalloc(&c->seeds[1], c->nc3);
    if (!e) e = dalloc(&c->coarse, c->nc3);
    if (!e) e = dalloc(&c->accum, c->nf3);
    if (!e) e = dalloc(&c->counts, c->nf3);
    if (!e) e = dalloc(&c->fine, c->nf3);
    if (!e) e = dalloc(&c->masked, c->nc3);
    if (!e) e = dalloc(&c->ray_min, 8 * c->nc3);
    if (!e) e = dalloc(&c->ray_cnt, 8 * c->nc3);
    if (!e) e = dalloc(&c->d_next_ray, 1);
    {
        const size_t g = (size_t)(c->nc + 7) / 8, cells = g * g * g;
        c->bin_cap = 1u << 23;
        if (!e) e = dalloc(&c->bin_count, cells);
        if (!e) e = dalloc(&c->bin_start, cells + 1);
        if (!e) e = dalloc(&c->bin_cursor, cells);
        if (!e) e = dalloc(&c->bin_items, (size_t)c->bin_cap);
        if (!e) e = dalloc(&c->bin_overflow, 1);
        if (!e) e = cudaMemsetAsync(c->bin_overflow, 0, sizeof(uint32_t), c->stream);
    }
    if (!e) e = dalloc(&c->d_masked_count, 1);
    if (!e) e = dalloc(&c->d_big_count, 1);
    if (!e) e = dalloc(&c->d_moved_count, 1);
    if (!e) e = dalloc(&c->d_err, 1);
    if (!e) e = dalloc(&c->d_counters, 1);
    if (!e) e = cudaMemsetAsync(c->d_counters, 0, sizeof(TraceCounters), c->stream);
    if (!e) e = cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->d_masked_count, 0, sizeof(uint32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->d_moved_count, 0, sizeof(int32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->seeds[0], 0xFF, c->nc3 * sizeof(uint32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->seeds[1], 0xFF, c->nc3 * sizeof(uint32_t), c->stream);
    if (!e) e = fill_f32(c, c->coarse, c->nc3, INFINITY);
    if (!e) e = fill_f32(c, reinterpret_cast<float*>(c->ray_min), 8 * c->nc3, INFINITY);
    if (!e) e = cudaMemsetAsync(c->ray_cnt, 0, 8 * c->nc3 * sizeof(uint32_t), c->stream);
    if (!e) e = reset_temporal(c);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        rtsdf_status s = from_cuda(e);
        free_all(c);
        delete c;
        return s;
    }
    *out = c;
    return RTSDF_OK;
}

rtsdf_status rtsdf_destroy(rtsdf_t c) {
    if (!c) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return RTSDF_OK;
}

rtsdf_status rtsdf_set_stream(rtsdf_t c, void* stream) {
    if (!c) return RTSDF_E_ARG;
    // work already enqueued on the old stream finishes first, so that later
    // calls on the new one are ordered after it (and no buffer or texture
    // object is released while that work may still use it)
    if ((cudaStream_t)stream != c->stream) {
        DeviceGuard g(c->device);
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    c->stream = (cudaStream_t)stream;
    c->cfg.stream = stream;
    return RTSDF_OK;
}

rtsdf_status rtsdf_upload_mesh(rtsdf_t c, const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                               int on_device) {
    if (!c || nv < 0 || nt < 0 || nv > INT32_MAX || nt > INT32_MAX / 3) return RTSDF_E_ARG;
    if ((nv > 0 && !verts) || (nt > 0 && !tris)) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) return from_cuda(e);
    // the old mesh is gone from here on, also when an allocation below fails
    c->have_mesh = false;
    c->nv = c->nt = 0;
    c->n_obj = 0;
    c->voxelized = c->flooded = false;
    c->bvh.built = false;
    c->bvh_dirty = true;
    c->reset_pending = false;
    if (nv > c->cap_v) {
        dfree(c->verts); dfree(c->qverts); dfree(c->vert_obj);
        c->cap_v = 0;
        if ((e = dalloc(&c->verts, 3 * nv)) || (e = dalloc(&c->qverts, 3 * nv))) return from_cuda(e);
        c->cap_v = nv;
    }
    if (nt > c->cap_t) {
        dfree(c->tris); dfree(c->big_list);
        c->cap_t = 0;
        if ((e = dalloc(&c->tris, 3 * nt)) || (e = dalloc(&c->big_list, nt))) return from_cuda(e);
        c->cap_t = nt;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nv > 0 && (e = cudaMemcpyAsync(c->verts, verts, sizeof(float) * 3 * nv, kind, c->stream))) return from_cuda(e);
    if (nt > 0 && (e = cudaMemcpyAsync(c->tris, tris, sizeof(int32_t) * 3 * nt, kind, c->stream))) return from_cuda(e);
    c->nv = nv;
    c->nt = nt;
    c->n_obj = 0;
    c->have_mesh = false;
    c->voxelized = c->flooded = false;
    c->bvh.built = false;
    c->bvh_dirty = true;
    c->reset_pending = false;
    if ((e = cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), c->stream))) return from_cuda(e);
    if ((e = launch_validate_tris(c))) return from_cuda(e);
    if ((e = launch_quantise(c))) return from_cuda(e);
    if ((e = reset_temporal(c))) return from_cuda(e);
    rtsdf_status s = sync_status(c);
    if (s != RTSDF_OK) return s;
    c->have_mesh = true;
    return RTSDF_OK;
}

rtsdf_status rtsdf_set_objects(rtsdf_t c, const int32_t* vert_object, int32_t n_objects, int on_device) {
    if (!c || n_objects < 1 || (c->nv > 0 && !vert_object)) return RTSDF_E_ARG;
    if (!c->have_mesh) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) return from_cuda(e);
    if (n_objects > c->cap_obj) {
        dfree(c->obj_box); dfree(c->obj_trans); dfree(c->obj_xform); dfree(c->moved_list);
        c->cap_obj = 0;
        if ((e = dalloc(&c->obj_box, 6 * (size_t)n_objects)) || (e = dalloc(&c->obj_trans, 3 * (size_t)n_objects)) ||
            (e = dalloc(&c->obj_xform, 12 * (size_t)n_objects)) || (e = dalloc(&c->moved_list, (size_t)n_objects)))
            return from_cuda(e);
        c->cap_obj = n_objects;
    }
    if (!c->vert_obj && (e = dalloc(&c->vert_obj, c->cap_v > 0 ? c->cap_v : 1))) return from_cuda(e);
    int32_t* tmp = nullptr;
    if ((e = dalloc(&tmp, c->nv > 0 ? c->nv : 1))) return from_cuda(e);
    if (c->nv > 0) {
        e = cudaMemcpyAsync(tmp, vert_object, sizeof(int32_t) * c->nv,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
        if (!e) {
            k_check_objects<<<(unsigned)((c->nv + 255) / 256), 256, 0, c->stream>>>(tmp, c->nv, n_objects, c->d_err,
                                                                                 c->vert_obj);
            c->launches++;
            e = cudaGetLastError();
        }
    }
    rtsdf_status s = e ? from_cuda(e) : sync_status(c);
    cudaFree(tmp);
    if (s != RTSDF_OK) return s;
    c->n_obj = n_objects;
    c->bvh.two_level = false;   // a two-level tree groups by the old objects: refits keep it whole
    return RTSDF_OK;
}

rtsdf_status rtsdf_move_objects(rtsdf_t c, const float* translations, int on_device) {
    if (!c || !translations) return RTSDF_E_ARG;
    if (!c->have_mesh || c->n_obj < 1) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_MOTION);
    cudaError_t e = cudaMemcpyAsync(c->obj_trans, translations, sizeof(float) * 3 * c->n_obj,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    if (!e) e = launch_move(c);
    if (!e) e = launch_quantise(c);
    if (e) return from_cuda(e);
    c->voxelized = c->flooded = false;
    c->bvh_dirty = true;
    c->reset_pending = c->reset_on;
    return RTSDF_OK;
}

rtsdf_status rtsdf_transform_objects(rtsdf_t c, const float* xforms, int on_device) {
    if (!c || !xforms) return RTSDF_E_ARG;
    if (!c->have_mesh || c->n_obj < 1) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_MOTION);
    cudaError_t e = cudaMemcpyAsync(c->obj_xform, xforms, sizeof(float) * 12 * c->n_obj,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    if (!e) e = launch_transform(c);
    if (!e) e = launch_quantise(c);
    if (e) return from_cuda(e);
    c->voxelized = c->flooded = false;
    c->bvh_dirty = true;
    c->reset_pending = c->reset_on;
    return RTSDF_OK;
}

rtsdf_status rtsdf_build_bvh(rtsdf_t c, int refit) {
    if (!c) return RTSDF_E_ARG;
    if (!c->have_mesh) return RTSDF_E_STATE;
    if (refit && (!c->bvh.built || c->bvh.nt != c->nt)) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_BVH);
    cudaError_t e = refit ? launch_bvh_refit(c) : launch_bvh_build(c);
    if (e) return from_cuda(e);
    c->bvh_dirty = false;
    return RTSDF_OK;
}

rtsdf_status rtsdf_voxelize(rtsdf_t c) {
    if (!c) return RTSDF_E_ARG;
    if (!c->have_mesh) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_VOX);
    cudaError_t e = launch_voxelize(c);
    if (e) return from_cuda(e);
    c->voxelized = true;
    c->flooded = false;
    return RTSDF_OK;
}

rtsdf_status rtsdf_jfa(rtsdf_t c) {
    if (!c) return RTSDF_E_ARG;
    if (!c->voxelized) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_JFA);
    cudaError_t e = launch_jfa(c);
    if (e) return from_cuda(e);
    c->flooded = true;
    return RTSDF_OK;
}

rtsdf_status rtsdf_trace(rtsdf_t c, float d_vox, int32_t rays, int32_t frame) {
    if (!c) return RTSDF_E_ARG;
    if (!isfinite(d_vox) || rays < 1 || rays > 1024 || (rays & (rays - 1)) || frame < 0) return RTSDF_E_ARG;
    if (!c->flooded || !c->bvh.built || c->bvh_dirty) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    cudaError_t e;
    {
        StageTimer tm(c, ST_MASK);
        e = launch_mask(c, d_vox);
    }
    if (e) return from_cuda(e);
    {
        StageTimer tm(c, ST_TRACE);
        e = launch_trace(c, rays, frame);
    }
    if (e) return from_cuda(e);
    c->last_masked = -1;
    return RTSDF_OK;
}

static rtsdf_status shadow_common(rtsdf_t c, const float* pos, const float* nrm, int64_t npix, const float light[3],
                                  float k, int32_t steps, float smax_vox, float eps_vox, float L[3], float* inv_norm) {
    if (!c || npix < 0 || (npix > 0 && (!pos || !nrm)) || !light) return RTSDF_E_ARG;
    if (steps < 1 || steps > MAX_SHADOW_STEPS || !(k > 0.f) || !isfinite(k)) return RTSDF_E_ARG;
    if (!(smax_vox > 0.f) || !isfinite(smax_vox) || !(eps_vox > 0.f) || !isfinite(eps_vox)) return RTSDF_E_ARG;
    if (!finite3(light)) return RTSDF_E_ARG;
    const double nv = sqrt((double)light[0] * light[0] + (double)light[1] * light[1] + (double)light[2] * light[2]);
    if (!(nv > 0)) return RTSDF_E_ARG;
    for (int a = 0; a < 3; a++) L[a] = (float)(light[a] / nv);
    *inv_norm = (float)(1.0 / nv);
    return RTSDF_OK;
}

rtsdf_status rtsdf_shadow(rtsdf_t c, const float* sdf, const float* pos, const float* nrm, int64_t npix,
                          const float light[3], float k, int32_t steps, float smax_vox, float eps_vox, float* vis) {
    float L[3], inv;
    rtsdf_status s = shadow_common(c, pos, nrm, npix, light, k, steps, smax_vox, eps_vox, L, &inv);
    if (s != RTSDF_OK) return s;
    if (npix > 0 && !vis) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_SHADOW);
    return from_cuda(launch_shadow(c, sdf, pos, nrm, npix, L, k, steps, smax_vox * c->hf, eps_vox * c->hf, 0.f, 0,
                                   vis));
}

rtsdf_status rtsdf_shadow_jittered(rtsdf_t c, const float* sdf, const float* pos, const float* nrm, int64_t npix,
                                   const float light[3], float k, int32_t steps, float smax_vox, float eps_vox,
                                   float jitter_vox, int32_t frame, float* vis) {
    float L[3], inv;
    rtsdf_status s = shadow_common(c, pos, nrm, npix, light, k, steps, smax_vox, eps_vox, L, &inv);
    if (s != RTSDF_OK) return s;
    if (npix > 0 && !vis) return RTSDF_E_ARG;
    if (!(jitter_vox >= 0.f) || !isfinite(jitter_vox) || frame < 0) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_SHADOW);
    return from_cuda(launch_shadow(c, sdf, pos, nrm, npix, L, k, steps, smax_vox * c->hf, eps_vox * c->hf,
                                   jitter_vox * c->hf, frame, vis));
}

rtsdf_status rtsdf_shadow_fallback(rtsdf_t c, const float* pos, const float* nrm, int64_t npix, const float light[3],
                                   float eps_vox, float* vis, uint8_t* blocked) {
    float L[3], inv;
    // k, steps, step_max are not used here: pass valid placeholders to the shared checks
    rtsdf_status s = shadow_common(c, pos, nrm, npix, light, 1.f, 1, 1.f, eps_vox, L, &inv);
    if (s != RTSDF_OK) return s;
    if (npix > 0 && !vis && !blocked) return RTSDF_E_ARG;
    if (!c->have_mesh || !c->bvh.built || c->bvh_dirty || c->bvh.nt != c->nt) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_SHADOW);
    return from_cuda(launch_shadow_exact(c, pos, nrm, npix, L, eps_vox * c->hf, vis, blocked));
}

rtsdf_status rtsdf_taa_resolve(rtsdf_t c, const float* cur, float* hist, int32_t width, int32_t height,
                               float blend) {
    if (!c || width < 0 || height < 0 || !(blend > 0.f && blend <= 1.f)) return RTSDF_E_ARG;
    const size_t bytes = (size_t)width * (size_t)height * sizeof(float);
    if (bytes == 0) return RTSDF_OK;
    if (!cur || !hist) return RTSDF_E_ARG;
    const char *a = reinterpret_cast<const char*>(cur), *b = reinterpret_cast<const char*>(hist);
    if (a < b + bytes && b < a + bytes) return RTSDF_E_ARG;   // in place only on the history
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_SHADOW);
    return from_cuda(launch_taa(c, cur, hist, width, height, blend));
}

rtsdf_status rtsdf_shadow_backward(rtsdf_t c, const float* sdf, const float* pos, const float* nrm, int64_t npix,
                                   const float light[3], float k, int32_t steps, float smax_vox, float eps_vox,
                                   const float* dvis, float* dsdf, float* dlight) {
    float L[3], inv;
    rtsdf_status s = shadow_common(c, pos, nrm, npix, light, k, steps, smax_vox, eps_vox, L, &inv);
    if (s != RTSDF_OK) return s;
    if (npix > 0 && (!dvis || !dsdf || !dlight)) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    StageTimer tm(c, ST_SHADOW_BWD);
    return from_cuda(launch_shadow_bwd(c, sdf, pos, nrm, npix, L, inv, k, steps, smax_vox * c->hf,
                                       eps_vox * c->hf, dvis, dsdf, dlight));
}

rtsdf_status rtsdf_get_grids(rtsdf_t c, rtsdf_grids* out) {
    if (!c || !out) return RTSDF_E_ARG;
    out->coarse_n = c->nc;
    out->fine_n = c->nf;
    out->seeds = c->seeds[c->cur];
    out->coarse = c->coarse;
    out->fine = c->fine;
    out->accum = c->accum;
    out->counts = c->counts;
    out->masked = c->masked;
    return RTSDF_OK;
}

rtsdf_status rtsdf_get_masked_count(rtsdf_t c, int64_t* n) {
    if (!c || !n) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    uint32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->d_masked_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return from_cuda(e);
    *n = v;
    c->last_masked = v;
    return RTSDF_OK;
}

rtsdf_status rtsdf_set_profiling(rtsdf_t c, int on) {
    if (!c) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    if (on && !c->timers[0].a[0]) {
        for (auto& t : c->timers)
            for (int i = 0; i < TIMER_RING; i++) {
                cudaError_t e = cudaEventCreate(&t.a[i]);
                if (!e) e = cudaEventCreate(&t.b[i]);
                if (e) return from_cuda(e);
            }
    }
    c->profiling = on != 0;
    return RTSDF_OK;
}

rtsdf_status rtsdf_set_counting(rtsdf_t c, int on) {
    if (!c) return RTSDF_E_ARG;
    c->counting = on != 0;
    return RTSDF_OK;
}

rtsdf_status rtsdf_get_stats(rtsdf_t c, rtsdf_stats* out) {
    if (!c || !out) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) return from_cuda(e);
    memset(out, 0, sizeof(*out));
    out->launches = c->launches;
    int64_t m = 0;
    if (rtsdf_get_masked_count(c, &m) == RTSDF_OK) out->n_masked_texels = 8 * m;
    out->jfa_passes = c->jfa_passes;
    out->bvh_depth = c->bvh.depth;
    for (int st = 0; st < ST_COUNT; st++) {
        Timer& t = c->timers[st];
        drain(t);
        out->stage_ms[st] = t.carry_ms;
        out->stage_calls[st] = t.carry_calls;
        t.carry_ms = 0.f;
        t.carry_calls = 0;
    }
    TraceCounters tc;
    e = cudaMemcpy(&tc, c->d_counters, sizeof(tc), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemset(c->d_counters, 0, sizeof(tc));
    if (e) return from_cuda(e);
    out->rays = (int64_t)tc.rays;
    out->node_visits = (int64_t)tc.visits;
    out->tri_tests = (int64_t)tc.tests;
    out->lane_slots = (int64_t)tc.slots;
    out->leaf_slots = (int64_t)tc.leaf_slots;
    return RTSDF_OK;
}

static const uint32_t STATE_MAGIC = 0x46445352u;   // "RSDF"

rtsdf_status rtsdf_state_size(rtsdf_t c, size_t* bytes) {
    if (!c || !bytes) return RTSDF_E_ARG;
    *bytes = 16 + c->nf3 * (sizeof(float) * 2 + sizeof(uint32_t));
    return RTSDF_OK;
}

rtsdf_status rtsdf_save_state(rtsdf_t c, void* host_buf, size_t bytes) {
    size_t need = 0;
    if (!c || !host_buf) return RTSDF_E_ARG;
    rtsdf_state_size(c, &need);
    if (bytes < need) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    uint8_t* p = (uint8_t*)host_buf;
    uint32_t hdr[4] = {STATE_MAGIC, 1u, (uint32_t)c->nc, (uint32_t)c->sign_mode};
    memcpy(p, hdr, 16);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (!e) e = cudaMemcpy(p + 16, c->accum, c->nf3 * sizeof(float), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(p + 16 + c->nf3 * 4, c->counts, c->nf3 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(p + 16 + c->nf3 * 8, c->fine, c->nf3 * sizeof(float), cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

rtsdf_status rtsdf_load_state(rtsdf_t c, const void* host_buf, size_t bytes) {
    size_t need = 0;
    if (!c || !host_buf) return RTSDF_E_ARG;
    rtsdf_state_size(c, &need);
    if (bytes < need) return RTSDF_E_ARG;
    const uint8_t* p = (const uint8_t*)host_buf;
    uint32_t hdr[4];
    memcpy(hdr, p, 16);
    if (hdr[0] != STATE_MAGIC || hdr[1] != 1u || hdr[2] != (uint32_t)c->nc) return RTSDF_E_ARG;
    if (hdr[3] != RTSDF_SIGN_VOTE && hdr[3] != RTSDF_SIGN_NEAREST) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (!e && (int)hdr[3] != c->sign_mode) {
        c->sign_mode = (int)hdr[3];   // the state carries its sign mode
        e = reset_scratch(c);
        if (!e) e = cudaStreamSynchronize(c->stream);
    }
    if (!e) e = cudaMemcpy(c->accum, p + 16, c->nf3 * sizeof(float), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(c->counts, p + 16 + c->nf3 * 4, c->nf3 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(c->fine, p + 16 + c->nf3 * 8, c->nf3 * sizeof(float), cudaMemcpyHostToDevice);
    return from_cuda(e);
}

rtsdf_status rtsdf_set_sign_mode(rtsdf_t c, int32_t mode) {
    if (!c || (mode != RTSDF_SIGN_VOTE && mode != RTSDF_SIGN_NEAREST)) return RTSDF_E_ARG;
    if (mode == c->sign_mode) return RTSDF_OK;
    DeviceGuard g(c->device);
    c->sign_mode = mode;
    cudaError_t e = reset_temporal(c);   // the counts word changes meaning: restart accumulation
    if (!e) e = reset_scratch(c);
    return from_cuda(e);
}

rtsdf_status rtsdf_get_sign_mode(rtsdf_t c, int32_t* mode) {
    if (!c || !mode) return RTSDF_E_ARG;
    *mode = c->sign_mode;
    return RTSDF_OK;
}

void rtsdf_debug_fail_allocation(int64_t after) { g_fail_after.store(after < 0 ? -1 : (long long)after); }

void rtsdf_debug_texture_fetch(int32_t on) { g_texture_fetch.store(on != 0); }

rtsdf_status rtsdf_debug_bvh_cycle(rtsdf_t c) {
    if (!c) return RTSDF_E_ARG;
    if (!c->bvh.built || c->bvh.n_wide < 1) return RTSDF_E_STATE;
    // the root is wide node 0; its child ids are one int4
    int4 ch;
    cudaError_t e = cudaMemcpyAsync(&ch, &c->bvh.wide[0].child, sizeof(int4), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return from_cuda(e);
    int* k = &ch.x;
    for (int i = 0; i < 4; i++)
        if (k[i] != WIDE_EMPTY) k[i] = 0;
    e = cudaMemcpyAsync(&c->bvh.wide[0].child, &ch, sizeof(int4), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? from_cuda(e) : RTSDF_OK;
}

rtsdf_status rtsdf_set_reset(rtsdf_t c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return RTSDF_E_ARG;
    c->reset_on = on != 0;
    if (!c->reset_on) c->reset_pending = false;
    return RTSDF_OK;
}

rtsdf_status rtsdf_get_reset(rtsdf_t c, int32_t* on) {
    if (!c || !on) return RTSDF_E_ARG;
    *on = c->reset_on ? 1 : 0;
    return RTSDF_OK;
}

rtsdf_status rtsdf_set_bvh_builder(rtsdf_t c, int32_t builder) {
    if (!c || (builder != RTSDF_BVH_LBVH && builder != RTSDF_BVH_SAH && builder != RTSDF_BVH_TWO_LEVEL))
        return RTSDF_E_ARG;
    c->bvh_builder = builder;
    return RTSDF_OK;
}

rtsdf_status rtsdf_get_bvh_builder(rtsdf_t c, int32_t* builder) {
    if (!c || !builder) return RTSDF_E_ARG;
    *builder = c->bvh_builder;
    return RTSDF_OK;
}

rtsdf_status rtsdf_get_bvh_topology(rtsdf_t c, int32_t* children, int32_t* leaf_tri, int32_t* root) {
    if (!c) return RTSDF_E_ARG;
    if (!c->bvh.built) return RTSDF_E_STATE;
    DeviceGuard g(c->device);
    const int64_t n = c->bvh.nt;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (!e && children && n > 1) {
        std::vector<BNode> nodes((size_t)(n - 1));
        e = cudaMemcpy(nodes.data(), c->bvh.nodes, sizeof(BNode) * (size_t)(n - 1), cudaMemcpyDeviceToHost);
        for (int64_t i = 0; !e && i < n - 1; i++) {
            children[2 * i] = nodes[(size_t)i].d.x;
            children[2 * i + 1] = nodes[(size_t)i].d.y;
        }
    }
    if (!e && leaf_tri && n > 0)
        e = cudaMemcpy(leaf_tri, c->bvh.leaf_tri, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost);
    if (!e && root) {
        *root = -1;
        if (n > 1) e = cudaMemcpy(root, c->bvh.root, sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    return from_cuda(e);
}

rtsdf_status rtsdf_sync(rtsdf_t c) {
    if (!c) return RTSDF_E_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaGetLastError();
    if (e) return from_cuda(e);
    return sync_status(c);
}

const char* rtsdf_status_str(rtsdf_status s) {
    switch (s) {
        case RTSDF_OK: return "ok";
        case RTSDF_E_ARG: return "invalid argument";
        case RTSDF_E_STATE: return "call out of order";
        case RTSDF_E_OOM: return "device allocation failed";
        case RTSDF_E_CUDA: return "CUDA error";
        case RTSDF_E_MESH: return "invalid mesh (index out of range, or vertex not finite / outside the accepted box)";
        case RTSDF_E_OVERFLOW: return "BVH traversal stack overflow";
        case RTSDF_E_TIMEOUT: return "bounded device wait expired";
    }
    return "unknown status";
}

const char* rtsdf_version(void) { return "0.1.0"; }

}  // extern "C"
