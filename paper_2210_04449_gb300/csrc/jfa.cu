// Sec. 2.1 -- 3D jump flooding of the voxel seeds, and the coarse SDF.
//
// Pass with step k: every voxel v reads the previous pass's nearest seed at
// the 27 voxels v + {-k, 0, k}^3 inside the grid and keeps the one with the
// smallest squared distance D2 to v, ties to the smaller packed value
// (= smaller linear index).  Steps are 2^(ceil(log2 N) - 1), ..., 2, 1.
// The last pass also writes the coarse SDF c = h_c sqrt(D2) - beta h_c.
//
// Seeds are packed bytes (x, y, z, 0).  The one-voxel-per-thread passes
// (jfa_dev.cuh) compute D2 with two byte dot products,
//   D2 = s.s - 2 s.v + v.v   (dp4a; wraps correctly modulo 2^32, D2 < 2^18),
// and push "no seed" (all ones) above every real distance by OR-ing the
// seed's top byte into D2; the z-blocked pass below shares the x/y part of
// D2 between the voxels of a column.  Either way the candidate key is the
// pair (D2, seed), compared lexicographically.
#include <math.h>
#include <math_constants.h>

#include <cuda.h>

#include <mutex>

#include "internal.cuh"
#include "jfa_dev.cuh"

namespace rtsdf {
namespace {

// Tiles of 32 x 8 voxels (x, y) per block, one z-plane per grid z.  The 27
// candidates are read branch-free: an offset that leaves the grid reads the
// voxel's own coordinate on that axis (always in bounds), a duplicate of
// another candidate of the set.  The arg-min runs in two passes over the 27
// (D2, seed) pairs kept in registers: the smallest D2 first, then the
// smallest seed among the candidates at that D2 -- the same result as a
// lexicographic (D2, seed) minimum.
template <bool FINAL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_jfa_pass(const uint32_t* __restrict__ in,
                                                     uint32_t* __restrict__ out, int n, int k,
                                                     float* __restrict__ coarse, float hc, float beta_h) {
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= n || y >= n) return;
    dev::jfa_voxel<FINAL, true>(in, out, n, k, x, y, z, coarse, hc, beta_h);
}

template <int TX, int TY>
void launch_pass(rtsdf_ctx* c, const uint32_t* in, uint32_t* out, int n, int k, bool final, float beta_h) {
    dim3 block(TX, TY, 1), grid((n + TX - 1) / TX, (n + TY - 1) / TY, n);
    if (final) RTSDF_LAUNCH(c, (k_jfa_pass<true, TX, TY>), grid, block, 0, in, out, n, k, c->coarse, c->hc, beta_h);
    else RTSDF_LAUNCH(c, (k_jfa_pass<false, TX, TY>), grid, block, 0, in, out, n, k, c->coarse, c->hc, beta_h);
}

// z-blocked pass (dev::jfa_zblock_column): blocks of 32 x 4 threads in
// (x, y), blockIdx.z = g k + rz.
template <bool FINAL, int T>
__global__ void __launch_bounds__(128, 4) k_jfa_zblock(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                      int n, int k, float* __restrict__ coarse, float hc,
                                                      float beta_h) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 4 + threadIdx.y;
    const int rz = (int)(blockIdx.z % (unsigned)k), g = (int)(blockIdx.z / (unsigned)k);
    if (x >= n || y >= n) return;
    dev::jfa_zblock_column<FINAL, T>(in, out, n, k, x, y, rz, g, coarse, hc, beta_h);
}

template <int T>
void launch_zblock(rtsdf_ctx* c, const uint32_t* in, uint32_t* out, int n, int k, bool final, float beta_h) {
    const int lat = (n + k - 1) / k;          // z-lattice members of the fullest residue class
    const int groups = (lat + T - 1) / T;
    dim3 block(32, 4, 1), grid((n + 31) / 32, (n + 3) / 4, (unsigned)(groups * k));
    if (final) RTSDF_LAUNCH(c, (k_jfa_zblock<true, T>), grid, block, 0, in, out, n, k, c->coarse, c->hc, beta_h);
    else RTSDF_LAUNCH(c, (k_jfa_zblock<false, T>), grid, block, 0, in, out, n, k, c->coarse, c->hc, beta_h);
}

// Coarse SDF without a pass (N = 1: no jump steps).
__global__ void k_coarse_only(const uint32_t* __restrict__ seeds, size_t n3, int n, float* __restrict__ coarse,
                              float hc, float beta_h) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const uint32_t x = i % n, y = (i / n) % n, z = i / ((size_t)n * n);
    const uint32_t v = pack_seed(x, y, z);
    const uint32_t s = seeds[i];
    coarse[i] = dev::coarse_value(s, dev::seed_d2(s, v, __dp4a(v, v, 0u)), hc, beta_h);
}

}  // namespace

cudaError_t launch_jfa(rtsdf_ctx* c) {
    const int n = c->nc;
    int L = 0;
    while ((1 << L) < n) L++;
    const float beta_h = c->cfg.beta_vox * c->hc;
    int passes = 0;
    for (int k = L > 0 ? (1 << (L - 1)) : 0; k >= 1; k >>= 1) {
        const uint32_t* in = c->seeds[c->cur];
        uint32_t* out = c->seeds[c->cur ^ 1];
        switch (c->tune.jfa_tile) {
            case 1: launch_pass<64, 4>(c, in, out, n, k, k == 1, beta_h); break;
            case 2: launch_pass<128, 2>(c, in, out, n, k, k == 1, beta_h); break;
            case 3: launch_pass<32, 4>(c, in, out, n, k, k == 1, beta_h); break;
            case 4: {
                const int lat = (n + k - 1) / k;
                if (lat <= 2) launch_zblock<2>(c, in, out, n, k, k == 1, beta_h);
                else if (lat <= 4) launch_zblock<4>(c, in, out, n, k, k == 1, beta_h);
                else launch_zblock<8>(c, in, out, n, k, k == 1, beta_h);
                break;
            }
            default: launch_pass<32, 8>(c, in, out, n, k, k == 1, beta_h); break;
        }
        c->cur ^= 1;
        passes++;
    }
    if (passes == 0)
        RTSDF_LAUNCH(c, k_coarse_only, (unsigned)((c->nc3 + 255) / 256), 256, 0, c->seeds[c->cur], c->nc3, n,
                     c->coarse, c->hc, beta_h);
    c->jfa_passes = passes;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free jump flood (rtsdf_jfa_noalloc).
//
// Hosts that manage every byte of device memory themselves -- an engine
// plug-in living inside another application's memory budget, or a render
// loop that forbids allocations after start-up because cudaMalloc/cudaFree
// can synchronise the device -- cannot let the library allocate.  This entry
// point runs the same passes as rtsdf_jfa on caller buffers; its only
// scratch (the second ping-pong grid) is the fixed array below, which every
// GPU that loads the library holds until the process exits.  Calls share the
// array, so calls that overlap on the GPU race; every pass rewrites the part
// of it that the next pass reads, so nothing needs clearing between calls.
// ---------------------------------------------------------------------------

namespace {

constexpr int NOALLOC_MAX_N = 128;             // 128^3 x 4 B = 8 MiB of scratch
constexpr int NOALLOC_CACHE = 64;              // contexts remembered

static __device__ __align__(256) uint32_t g_jfa_scratch[NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N];

// The array's device address differs between CUDA contexts (each context
// loads its own copy of the module), so it is remembered per context, keyed
// by the context's unique id (cuCtxGetId: never reused within a process, so
// a context created after cudaDeviceReset gets a fresh lookup even if its
// handle value repeats).  The two driver calls are resolved through the
// runtime, so the library does not link libcuda itself.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

std::mutex g_scratch_mutex;
PfnCtxGetCurrent g_ctx_current = nullptr;
PfnCtxGetId g_ctx_id = nullptr;
bool g_driver_resolved = false;
unsigned long long g_cache_id[NOALLOC_CACHE] = {};
uint32_t* g_cache_ptr[NOALLOC_CACHE] = {};
int g_cache_n = 0, g_cache_next = 0;

void resolve_driver_calls() {
    if (g_driver_resolved) return;
    g_driver_resolved = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_current = reinterpret_cast<PfnCtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_id = reinterpret_cast<PfnCtxGetId>(f);
}

// Device address of the scratch array in the current context.  The lookup
// (cudaGetSymbolAddress, with the caller's device and context current) runs
// once per context; without a current context, or if the driver calls are
// unavailable, it runs on every call (the runtime then makes the device's
// primary context current).
cudaError_t scratch_for_current_context(uint32_t** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    resolve_driver_calls();
    unsigned long long id = 0;
    bool keyed = false;
    CUcontext ctx = nullptr;
    if (g_ctx_current && g_ctx_id && g_ctx_current(&ctx) == CUDA_SUCCESS && ctx != nullptr &&
        g_ctx_id(ctx, &id) == CUDA_SUCCESS)
        keyed = true;
    if (keyed)
        for (int i = 0; i < g_cache_n; i++)
            if (g_cache_id[i] == id) {
                *out = g_cache_ptr[i];
                return cudaSuccess;
            }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_jfa_scratch);
    if (e != cudaSuccess) return e;
    if (keyed) {
        g_cache_id[g_cache_next] = id;
        g_cache_ptr[g_cache_next] = static_cast<uint32_t*>(p);
        g_cache_next = (g_cache_next + 1) % NOALLOC_CACHE;
        if (g_cache_n < NOALLOC_CACHE) g_cache_n++;
    }
    *out = static_cast<uint32_t*>(p);
    return cudaSuccess;
}

__global__ void k_copy_u32(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

}  // namespace rtsdf

extern "C" rtsdf_status rtsdf_jfa_noalloc(const uint32_t* seeds_in, uint32_t* seeds_out, float* coarse_out,
                                          int32_t n, float extent, float beta_vox, void* stream) {
    using namespace rtsdf;
    if (!seeds_in || !seeds_out || !coarse_out) return RTSDF_E_ARG;
    if (n < 1 || n > NOALLOC_MAX_N) return RTSDF_E_ARG;
    if (!(extent > 0.f) || !isfinite(extent) || !(beta_vox >= 0.f) || !isfinite(beta_vox)) return RTSDF_E_ARG;
    const size_t n3 = (size_t)n * n * n;
    if (overlaps(seeds_in, n3 * 4, seeds_out, n3 * 4) || overlaps(seeds_in, n3 * 4, coarse_out, n3 * 4) ||
        overlaps(seeds_out, n3 * 4, coarse_out, n3 * 4))
        return RTSDF_E_ARG;
    uint32_t* scratch = nullptr;
    if (scratch_for_current_context(&scratch) != cudaSuccess) return RTSDF_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float hc = extent / (float)n;
    float beta_h = beta_vox * hc;
    int L = 0;
    while ((1 << L) < n) L++;
    // every launch goes through cudaLaunchKernel, whose return value is the
    // status of that launch alone (an error left pending by someone else's
    // earlier launch is neither reported nor cleared here)
    size_t nn = n3;
    int ni = n;
    if (L == 0) {
        const dim3 grid((unsigned)((n3 + 255) / 256)), block(256);
        void* a_copy[] = {(void*)&seeds_in, (void*)&seeds_out, (void*)&nn};
        if (cudaLaunchKernel((const void*)k_copy_u32, grid, block, a_copy, 0, s) != cudaSuccess) return RTSDF_E_CUDA;
        void* a_coarse[] = {(void*)&seeds_in, (void*)&nn, (void*)&ni, (void*)&coarse_out, (void*)&hc, (void*)&beta_h};
        if (cudaLaunchKernel((const void*)k_coarse_only, grid, block, a_coarse, 0, s) != cudaSuccess)
            return RTSDF_E_CUDA;
        return RTSDF_OK;
    }
    // pass i (1-based, L passes) writes seeds_out when L - i is even, else
    // the scratch array, so the last pass lands in seeds_out
    const dim3 block(32, 8, 1), grid((n + 31) / 32, (n + 7) / 8, n);
    const uint32_t* in = seeds_in;
    for (int i = 1; i <= L; i++) {
        int k = 1 << (L - i);
        uint32_t* out = ((L - i) % 2 == 0) ? seeds_out : scratch;
        void* args[] = {(void*)&in, (void*)&out, (void*)&ni, (void*)&k, (void*)&coarse_out, (void*)&hc, (void*)&beta_h};
        const void* fn = (i == L) ? (const void*)k_jfa_pass<true, 32, 8> : (const void*)k_jfa_pass<false, 32, 8>;
        if (cudaLaunchKernel(fn, grid, block, args, 0, s) != cudaSuccess) return RTSDF_E_CUDA;
        in = out;
    }
    return RTSDF_OK;
}
