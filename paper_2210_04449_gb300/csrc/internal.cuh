// Internal declarations shared by the CUDA translation units of librtsdf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rtsdf.h"

namespace rtsdf {

// Device status bits (accumulated with atomicOr, read by rtsdf_sync).
enum : uint32_t {
    ERR_MESH = 1u,
    ERR_STACK = 2u,
    ERR_TIMEOUT = 4u,
};

// Packed seed coordinate: x | y << 8 | z << 16 (N <= 256), EMPTY = all ones.
// Packed order equals linear-index order, so "smaller packed" is the
// smaller-linear-index tie-break of the jump flood.
constexpr uint32_t SEED_EMPTY = 0xFFFFFFFFu;
constexpr int QSUB = 256;          // vertex quantisation steps per coarse voxel
constexpr int MAX_N = 256;         // coarse voxels per axis
constexpr int TRACE_STACK = 64;    // BVH traversal stack depth per ray
constexpr int MAX_SHADOW_STEPS = 256;

__host__ __device__ inline uint32_t pack_seed(uint32_t x, uint32_t y, uint32_t z) {
    return x | (y << 8) | (z << 16);
}

// Binary BVH node: the two child boxes side by side (one 64-byte fetch
// decides both children).  Child index >= 0: internal node; < 0: ~leaf,
// where a leaf is a triangle position in Morton order.
struct __align__(16) BNode {
    float4 a;   // lo_l.x, hi_l.x, lo_l.y, hi_l.y
    float4 b;   // lo_r.x, hi_r.x, lo_r.y, hi_r.y
    float4 c;   // lo_l.z, hi_l.z, lo_r.z, hi_r.z
    int4 d;     // left, right, parent, unused
};

// 4-wide node collapsed from the binary tree: child boxes SoA (one float4
// per plane), child ids (>= 0 wide node, < 0 ~leaf), and for the refit the
// binary source of every child (>= 0 binary node, < 0 ~leaf, WIDE_EMPTY = no
// child; an empty slot has lo = +inf, hi = -inf and never hits).  128 bytes,
// 32-byte aligned: each (lo, hi) pair of an axis is one 32-byte sector.
// Leaf triangles: (v0, original index), e1, e2 as float4 and one float4 of
// padding, so that each triangle is two aligned 32-byte sectors.
constexpr int TRI_F4 = 4;
constexpr int WIDE_EMPTY = (int)0x80000000;
struct __align__(32) WNode {
    float4 lox, hix, loy, hiy, loz, hiz;
    int4 child;
    int4 src;
};
static_assert(sizeof(WNode) == 128, "4-wide node is 128 bytes");

struct Bvh {
    int64_t nt = 0;
    BNode* nodes = nullptr;        // [nt - 1]
    WNode* wide = nullptr;         // [n_wide] (capacity wide_cap = nt - 1)
    int64_t wide_cap = 0;
    // device collapse scratch: frontier (binary node, wide slot) x 2, kids, counts
    int32_t *col_fb = nullptr, *col_fslot = nullptr, *col_nb = nullptr, *col_nslot = nullptr;
    int4* col_kids = nullptr;
    uint32_t* col_nint = nullptr;
    int32_t* col_total = nullptr;
    int64_t col_cap = 0;
    int64_t n_wide = 0;
    cudaTextureObject_t wtex = 0;  // the wide nodes as int4 texels (0: none; see make_int4_texture)
    float* nbox = nullptr;         // [nt - 1][6] box of every binary node
    float* lbox = nullptr;         // [nt][6] padded box of every leaf
    float4* tri = nullptr;         // [3 nt] per leaf: (v0, orig idx bits), (e1, 0), (e2, 0)
    int32_t* leaf_tri = nullptr;   // [nt] original triangle index of each leaf
    int32_t* leaf_parent = nullptr;// [nt]
    uint32_t* flags = nullptr;     // [nt] bottom-up visit counters
    int32_t* root = nullptr;       // [1] binary root node (device)
    int64_t cap_nt = 0;            // capacity of the per-triangle arrays above
    // build scratch, kept across builds: Morton keys / order x 2, radix
    // histograms, depth, and the SAH builder's arena
    uint32_t *mk0 = nullptr, *mk1 = nullptr, *hist = nullptr;
    int32_t *mv0 = nullptr, *mv1 = nullptr, *d_depth = nullptr;
    void* sah = nullptr;
    size_t sah_bytes = 0;
    // two-level form (RTSDF_BVH_TWO_LEVEL): one subtree per object, kept
    // across frames, under a top tree over the objects that every refit
    // rebuilds
    bool two_level = false;
    int32_t top_n = 0;              // objects with triangles (listed in object order)
    int32_t top_cap = 0;
    int32_t* top_child = nullptr;   // [top_n] subtree of each listed object (node id or ~leaf)
    int32_t* top_ids = nullptr;     // [top_n - 1] node ids of the top tree
    float4* top_box = nullptr;      // [2 top_n] box (lo, hi) of each listed object
    void* top_scratch = nullptr;    // sah_top's arena
    int32_t* obj_count = nullptr;   // [n_obj] triangles per object (build scratch)
    int32_t obj_cap = 0;
    int depth = 0;
    bool built = false;
};

// Binned-SAH topology (bvh_sah.cu): fills nodes[].d, leaf_parent, *root and
// order[] (triangle at each leaf position) for nt >= 2.
size_t sah_scratch_bytes(int64_t nt);
cudaError_t sah_topology(rtsdf_ctx* c, void* scratch, int32_t* order);
// One subtree per segment [bounds[k], bounds[k+1]) of the leaf positions
// (order_in: triangle at each position; bounds: host [nseg + 1]); the
// subtree of segment k is hooked at seg_root[k] (device), its root's parent
// left negative.  order may not alias order_in.
cudaError_t sah_segments(rtsdf_ctx* c, void* scratch, int32_t* order, const int32_t* order_in,
                         const int32_t* bounds, int32_t nseg, int32_t* seg_root);
// Top tree over 1 <= nseg <= 1024 subtrees: boxes (lo, hi per subtree),
// node ids [nseg - 1], child_of [nseg]; hooks the subtrees' parents and the
// root.  scratch: sah_top_bytes(nseg), prepared by sah_top_prepare.
size_t sah_top_bytes(int32_t nseg);
cudaError_t sah_top_prepare(rtsdf_ctx* c, void* scratch, int32_t nseg);
cudaError_t sah_top(rtsdf_ctx* c, void* scratch, int32_t nseg, const float4* boxes, const int32_t* node_ids,
                    const int32_t* child_of);
constexpr int SAH_TOP_MAX = 1024;

// Ring of event pairs per stage; summed (and emptied) by rtsdf_get_stats.
constexpr int TIMER_RING = 128;
struct Timer {
    cudaEvent_t a[TIMER_RING] = {}, b[TIMER_RING] = {};
    int n = 0;          // recorded pairs not yet summed
    float carry_ms = 0; // sums of pairs drained early (ring full)
    int carry_calls = 0;
};

enum Stage { ST_VOX, ST_JFA, ST_MASK, ST_TRACE, ST_BVH, ST_SHADOW, ST_SHADOW_BWD, ST_MOTION, ST_COUNT };

// tracer work counters (device): rays, node visits, triangle tests
struct TraceCounters {
    unsigned long long rays, visits, tests;
    unsigned long long slots, leaf_slots;   // lane slots of the traversal iterations / of its leaf phases
};

}  // namespace rtsdf

struct rtsdf_ctx {
    rtsdf_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0;
    int nc = 0, nf = 0;
    size_t nc3 = 0, nf3 = 0;
    float hc = 0.f, hf = 0.f;

    // mesh
    float* verts = nullptr;       // [nv * 3] current positions
    int32_t* qverts = nullptr;    // [nv * 3] quantised positions
    int32_t* tris = nullptr;      // [nt * 3]
    int64_t nv = 0, nt = 0, cap_v = 0, cap_t = 0;
    bool have_mesh = false;

    // rigid objects
    int32_t* vert_obj = nullptr;  // [nv]
    int n_obj = 0, cap_obj = 0;
    float* obj_box = nullptr;     // [n_obj * 6] box before the last move (lo xyz, hi xyz)
    float* obj_trans = nullptr;   // [n_obj * 3]
    float* obj_xform = nullptr;   // [n_obj * 12] rigid transforms (rtsdf_transform_objects), rows of [R | t]
    int32_t* moved_list = nullptr;// [n_obj] objects with a non-zero translation
    int32_t* d_moved_count = nullptr;
    bool reset_pending = false;
    bool reset_on = true;         // rtsdf_set_reset: moves schedule the reset in changed regions
    // moved boxes binned on a coarse cell grid for the reset test
    uint32_t* bin_count = nullptr;
    uint32_t* bin_start = nullptr;
    uint32_t* bin_cursor = nullptr;
    int32_t* bin_items = nullptr;
    uint32_t* bin_overflow = nullptr;
    uint32_t bin_cap = 0;

    // coarse grid
    uint32_t* seeds[2] = {nullptr, nullptr};
    int cur = 0;                  // seeds[cur] holds the latest result
    float* coarse = nullptr;
    bool voxelized = false, flooded = false;
    int jfa_passes = 0;

    // voxelization work list of large triangles
    int32_t* big_list = nullptr;
    uint32_t* d_big_count = nullptr;

    // fine grid
    float* accum = nullptr;
    uint32_t* counts = nullptr;
    float* fine = nullptr;
    uint32_t* masked = nullptr;   // masked coarse voxels
    uint32_t* d_masked_count = nullptr;
    int64_t last_masked = -1;

    // tracer scratch: per texel slot (8 per masked voxel) this frame's
    // smallest hit distance (float bits, +inf = none) and front | back << 16
    // hit counts; cleared again by the finalize kernel
    uint32_t* ray_min = nullptr;
    uint32_t* ray_cnt = nullptr;
    unsigned long long* d_next_ray = nullptr;
    unsigned trace_grid = 0;

    // launch parameters (rtsdf_set_tuning / rtsdf_autotune)
    int sign_mode = RTSDF_SIGN_VOTE;   // rtsdf_set_sign_mode
    int bvh_builder = RTSDF_BVH_SAH;   // rtsdf_set_bvh_builder
    rtsdf_tuning tune = {4, 0, 12, 1024, 12};   // the autotuner's usual pick

    rtsdf::Bvh bvh;
    bool bvh_dirty = true;

    uint32_t* d_err = nullptr;
    int64_t launches = 0;
    bool profiling = false;
    bool counting = false;
    rtsdf::TraceCounters* d_counters = nullptr;
    rtsdf::Timer timers[rtsdf::ST_COUNT];
};

namespace rtsdf {

// Launch helpers (count every kernel this context launches).
#define RTSDF_LAUNCH(ctx, kern, grid, block, smem, ...)                       \
    do {                                                                      \
        kern<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);        \
        (ctx)->launches++;                                                    \
    } while (0)

// Stage launchers, one per translation unit; each returns a cudaError_t of
// the launches (cudaGetLastError), never synchronises.
cudaError_t launch_quantise(rtsdf_ctx* c);
cudaError_t launch_validate_tris(rtsdf_ctx* c);
cudaError_t launch_voxelize(rtsdf_ctx* c);
cudaError_t launch_jfa(rtsdf_ctx* c);
cudaError_t launch_mask(rtsdf_ctx* c, float d_vox);
cudaError_t launch_trace(rtsdf_ctx* c, int rays, int frame);
// A texture object over `count` int4 texels at `ptr` (raw 32-bit words), or
// 0 when the array exceeds the device's linear-texture width or creation
// fails (the traversal then reads the nodes with plain loads).  drop_texture
// destroys one; the caller makes sure no launch still uses it.
cudaTextureObject_t make_int4_texture(const void* ptr, size_t count, int device);
void drop_texture(cudaTextureObject_t& t);
// Whether launches may take the texture path (rtsdf_debug_texture_fetch).
bool texture_fetch_on();
cudaError_t launch_bvh_build(rtsdf_ctx* c);
cudaError_t launch_bvh_refit(rtsdf_ctx* c);
cudaError_t launch_move(rtsdf_ctx* c);
cudaError_t launch_transform(rtsdf_ctx* c);
cudaError_t launch_shadow(rtsdf_ctx* c, const float* sdf, const float* pos, const float* nrm,
                          int64_t npix, const float L[3], float k, int steps, float smax,
                          float eps, float jitter, int frame, float* vis);
cudaError_t launch_taa(rtsdf_ctx* c, const float* cur, float* hist, int w, int h, float blend);
cudaError_t launch_shadow_exact(rtsdf_ctx* c, const float* pos, const float* nrm, int64_t npix, const float L[3],
                                float eps, float* vis, uint8_t* blocked);
cudaError_t launch_shadow_bwd(rtsdf_ctx* c, const float* sdf, const float* pos, const float* nrm,
                              int64_t npix, const float L[3], float inv_norm, float k, int steps,
                              float smax, float eps, const float* dvis, float* dsdf,
                              float* dlight);

// Resident blocks per SM of the per-scene tracer kernel.
cudaError_t trace_occupancy(int* per_sm);

// Mask threshold T = floor((d + beta)^2) in coarse voxels (-1: nothing masked).
int64_t mask_threshold(float d_vox, float beta_vox);

}  // namespace rtsdf
