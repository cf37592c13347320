/*
 * rtsdf.h -- C ABI of the GB300 (sm_103a) real-time SDF generator.
 *
 * Implements the method of "RTSDF: Generating Signed Distance Fields in Real
 * Time for Soft Shadow Rendering" (Tan, Chua, Koh, Bhojan, Pacific Graphics
 * 2020): a coarse SDF by voxelization and 3D jump flooding (Sec. 2.1), a
 * fine SDF by ray tracing fine texels near surfaces with temporal
 * accumulation (Sec. 2.2, Eq. 1), and soft shadows by sphere tracing the fine
 * SDF (Sec. 2.3), plus the reverse-mode derivative of the shadow pass.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grids.  The scene bounds are the cube [bmin, bmin + extent]^3.  The coarse
 *   grid has N = coarse_n voxels per axis (1 <= N <= 256), voxel size
 *   h_c = extent / N; the fine grid has 2N texels per axis, h_f = h_c / 2.
 *   Every grid is stored x-fastest: element (x, y, z) at x + n*(y + n*z).
 *   A voxel/texel value describes its centre, bmin + (i + 0.5) * h.
 * Streams.  Every call that launches work enqueues it on the context's
 *   stream (rtsdf_config.stream / rtsdf_set_stream) and returns without
 *   waiting, except where a call says it synchronises.
 * Memory.  The library allocates and owns all grids, the mesh copy and the
 *   BVH (cudaMalloc at creation / upload, cudaFree at destroy).  Caller
 *   buffers (G-buffers, outputs, gradients) are caller-owned device pointers
 *   that must stay valid until the enqueued work has finished.
 * Errors.  Argument and ordering errors are reported synchronously by the
 *   return value.  Errors found by device code (invalid mesh data found
 *   after upload, a BVH traversal stack overflow) set a device status word
 *   that the next rtsdf_sync() returns (and clears).  The library never
 *   aborts, traps or prints.
 * Threads.  A context must not be used from two host threads at once;
 *   distinct contexts are independent.
 */
#ifndef RTSDF_H
#define RTSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtsdf_ctx* rtsdf_t;

typedef enum {
    RTSDF_OK = 0,
    RTSDF_E_ARG = 1,       /* invalid argument: null pointer, size or value out of range */
    RTSDF_E_STATE = 2,     /* call out of order (e.g. rtsdf_jfa before rtsdf_voxelize) */
    RTSDF_E_OOM = 3,       /* device allocation failed */
    RTSDF_E_CUDA = 4,      /* CUDA runtime error (launch failure, sticky device error) */
    RTSDF_E_MESH = 5,      /* triangle index out of range, or a vertex not finite or
                              outside [bmin - extent/2, bmin + 3 extent/2]^3 */
    RTSDF_E_OVERFLOW = 6,  /* a BVH traversal exceeded its fixed stack or its step bound (result incomplete) */
    RTSDF_E_TIMEOUT = 7    /* a bounded device-side wait expired (batched form) */
} rtsdf_status;

typedef struct {
    float bmin[3];      /* lower corner of the scene cube */
    float extent;       /* edge length of the scene cube, > 0 */
    int32_t coarse_n;   /* coarse voxels per axis, 1..256; fine grid = 2 * coarse_n */
    float beta_vox;     /* Sec. 2.1 bias beta, in coarse voxels (>= 0) */
    float alpha;        /* Eq. 1 decay alpha in [0, 1]; 1 = plain temporal minimum */
    uint64_t seed;      /* key of the Philox stream for the ray directions */
    void* stream;       /* cudaStream_t to enqueue on; NULL = legacy default stream */
} rtsdf_config;

/* Device pointers into the context's grids (borrowed: valid until the next
 * call that reallocates them, i.e. rtsdf_destroy). */
typedef struct {
    int32_t coarse_n, fine_n;
    const uint32_t* seeds;   /* [coarse_n^3] nearest seed after rtsdf_jfa, packed
                                x | y << 8 | z << 16; 0xFFFFFFFF = no seed */
    const float* coarse;     /* [coarse_n^3] coarse SDF c = h_c (sqrt(D2) - beta); +inf = no seed */
    const float* fine;       /* [fine_n^3] signed fine SDF f_t (Eq. 1 and the sign vote) */
    const float* accum;      /* [fine_n^3] unsigned accumulator u_t of traced texels; +inf = none */
    const uint32_t* counts;  /* [fine_n^3] front-hit count | back-hit count << 16 (saturating) */
    const uint32_t* masked;  /* [n_masked_coarse] coarse voxels whose 8 fine texels were traced */
} rtsdf_grids;

/* Pipeline stages, in the order of rtsdf_stats.stage_ms / stage_calls. */
typedef enum {
    RTSDF_STAGE_VOXELIZE = 0, RTSDF_STAGE_JFA = 1, RTSDF_STAGE_MASK = 2, RTSDF_STAGE_TRACE = 3,
    RTSDF_STAGE_BVH = 4, RTSDF_STAGE_SHADOW = 5, RTSDF_STAGE_SHADOW_BWD = 6, RTSDF_STAGE_MOTION = 7,
    RTSDF_STAGE_COUNT = 8
} rtsdf_stage;

typedef struct {
    int64_t launches;         /* kernels launched by this context since creation */
    int64_t n_masked_texels;  /* fine texels traced by the last rtsdf_trace (8 per masked voxel) */
    int32_t jfa_passes;       /* passes run by the last rtsdf_jfa */
    int32_t bvh_depth;        /* depth of the BVH (0 before the first build) */
    /* Device time (CUDA events on the context stream) summed over the calls
       of each stage since the previous rtsdf_get_stats, and the number of
       those calls; only while profiling is on (rtsdf_set_profiling). */
    float stage_ms[RTSDF_STAGE_COUNT];
    int32_t stage_calls[RTSDF_STAGE_COUNT];
    /* Tracer work since the previous rtsdf_get_stats, only while counting is
       on (rtsdf_set_counting): rays cast, BVH nodes entered, ray/triangle
       tests (node_visits includes them); and the SIMT use of the traversal
       loop: lane slots (32 per warp and node step) of its node steps, and
       lane slots (32 per warp and round) of its triangle rounds (a triangle
       phase runs one round, or two when enough lanes reach a second leaf).
       Lanes busy per node step = (node_visits - tri_tests) / lane_slots x 32,
       per triangle round = tri_tests / leaf_slots x 32. */
    int64_t rays, node_visits, tri_tests;
    int64_t lane_slots, leaf_slots;
} rtsdf_stats;

/* Sec. 2: create a context (allocates both grids on the current device).
 * Returns RTSDF_E_ARG for an invalid config, RTSDF_E_OOM when the grids do
 * not fit. */
rtsdf_status rtsdf_create(const rtsdf_config* cfg, rtsdf_t* out);

/* Frees every device buffer of the context (synchronises its stream first). */
rtsdf_status rtsdf_destroy(rtsdf_t ctx);

/* Changes the stream later calls enqueue on.  Waits first for the work
 * already enqueued on the previous stream (RTSDF_E_CUDA if that work
 * failed), so later calls are ordered after it. */
rtsdf_status rtsdf_set_stream(rtsdf_t ctx, void* stream);

/* Sec. 2.1 input: copy a triangle mesh into the context.  verts: float32
 * [nv, 3]; tris: int32 [nt, 3] (counter-clockwise seen from outside = front
 * face).  on_device != 0: both pointers are device pointers, else host.
 * Validates the data (synchronises) and returns RTSDF_E_MESH for an index
 * outside [0, nv) or a vertex that is not finite or lies outside
 * [bmin - extent/2, bmin + 3 extent/2]^3.  nt = 0 is an empty scene.
 * Resets the accumulated fine SDF and invalidates the BVH. */
rtsdf_status rtsdf_upload_mesh(rtsdf_t ctx, const float* verts, int64_t nv,
                               const int32_t* tris, int64_t nt, int on_device);

/* Rigid objects for animated scenes: vert_object int32 [nv] gives each
 * vertex's object id in [0, n_objects).  Host or device pointer. */
rtsdf_status rtsdf_set_objects(rtsdf_t ctx, const int32_t* vert_object, int32_t n_objects,
                               int on_device);

/* Moves every object by its translation (float32 [n_objects, 3], host or
 * device pointer): v += t[object(v)] in fp32.  Records the previous
 * bounding box of every object with a non-zero translation; the next
 * rtsdf_trace restarts the accumulation of traced texels whose centre lies
 * within their accumulated distance of such a box (reset in changed
 * regions).  Vertices that leave the accepted box set RTSDF_E_MESH at the
 * next rtsdf_sync and are clamped. */
rtsdf_status rtsdf_move_objects(rtsdf_t ctx, const float* translations, int on_device);

/* Moves every object by a rigid transform (float32 [n_objects][3][4], rows
 * of [R | t], host or device pointer): v' = R v + t in fp32 with each
 * product and sum rounded in the order v'_a = ((R_a0 x + R_a1 y) + R_a2 z)
 * + t_a (no fused multiply-add), so a caller can reproduce the positions
 * exactly.  An object whose transform is exactly the identity does not
 * move; the others are handled as in rtsdf_move_objects (their previous
 * bounding boxes drive the reset in changed regions at the next trace).
 * Vertices that leave the accepted box set RTSDF_E_MESH at the next
 * rtsdf_sync and are clamped. */
rtsdf_status rtsdf_transform_objects(rtsdf_t ctx, const float* xforms, int on_device);

/* Reset in changed regions on (1, default) or off (0).  The paper keeps
 * moving objects' old distances from persisting only through the temporal
 * weight alpha of Eq. 1 (Sec. 2.2); with the reset off, moves leave the
 * accumulation alone and alpha < 1 is what lets stale minima fade.
 * Turning it off drops a reset already scheduled by a move.  RTSDF_E_ARG
 * for any other value. */
rtsdf_status rtsdf_set_reset(rtsdf_t ctx, int32_t on);
rtsdf_status rtsdf_get_reset(rtsdf_t ctx, int32_t* on);

/* Test hook for the allocation-failure paths (not a step of the paper):
 * after `after` more device allocations of a context (grids, mesh, BVH and
 * tracer buffers) succeed, the next one fails as if the device were out of
 * memory, without calling the allocator; the call that made it returns
 * RTSDF_E_OOM, frees what it had allocated, and the hook turns itself off.
 * after < 0 turns it off.  Process-wide; for tests only. */
void rtsdf_debug_fail_allocation(int64_t after);

/* Test hook for the traversal's bounded-error path (not a step of the
 * paper): rewrites the child ids of the context's root BVH node so that
 * every non-empty child names the root itself -- a valid node index that
 * closes a cycle.  A traversal that enters the cycle stops at its per-ray
 * step bound (node and leaf steps <= 2 T + 2 for T triangles) or at its
 * stack limit, with every memory access in bounds, and the next sync
 * returns RTSDF_E_OVERFLOW.  A refit keeps the cycle (it keeps the
 * topology); the next full rtsdf_build_bvh(ctx, 0) writes a valid tree.
 * RTSDF_E_STATE without a built BVH over at least two triangles.  Waits for
 * the context's stream.  For tests only. */
rtsdf_status rtsdf_debug_bvh_cycle(rtsdf_t ctx);

/* Test switch for the tracers' node fetch (not a step of the paper): on
 * (the default) the BVH traversal takes part of each node through the
 * texture pipe when the node array fits a linear texture; off, every fetch
 * is a plain load (the path for arrays beyond the texture width).  Both give
 * the same results.  Process-wide, read at each launch; for tests only. */
void rtsdf_debug_texture_fetch(int32_t on);

/* Builds (refit = 0) a binary BVH over the uploaded triangles, one triangle
 * per leaf, collapsed to 4-wide nodes for the tracer, or recomputes its
 * boxes for the current vertex positions keeping the topology (refit = 1;
 * requires a build).  The topology comes from the context's builder
 * (rtsdf_set_bvh_builder).  Traced results do not depend on the tree: every
 * ray finds its closest hit (equal distances: smaller triangle index). */
rtsdf_status rtsdf_build_bvh(rtsdf_t ctx, int refit);

/* Topology of the next full build.
 * RTSDF_BVH_SAH (default): top-down binned surface-area heuristic (32 bins
 *   of the centroid bounds per axis; ranges of <= 32 triangles split at the
 *   exact minimum over the centroids sorted along each axis).  About 13 %
 *   fewer node visits per ray than the Morton tree, a slower build.
 * RTSDF_BVH_LBVH: Karras' radix tree over 30-bit Morton codes of the
 *   centroids (fastest build).
 * RTSDF_BVH_TWO_LEVEL: for rigidly moving objects (rtsdf_set_objects): one
 *   SAH subtree per object (triangles grouped by their first vertex's
 *   object) under an SAH top tree over the objects.  A refit
 *   (rtsdf_build_bvh(ctx, 1)) refits the subtrees in world space and
 *   rebuilds the top tree, so the tree keeps its quality as objects move,
 *   for a fraction of a full build.  Without objects, or with more than 1024
 *   objects that own triangles, a build makes one SAH tree instead.
 * RTSDF_E_ARG for an unknown builder. */
typedef enum { RTSDF_BVH_LBVH = 0, RTSDF_BVH_SAH = 1, RTSDF_BVH_TWO_LEVEL = 2 } rtsdf_bvh_builder;
rtsdf_status rtsdf_set_bvh_builder(rtsdf_t ctx, int32_t builder);
rtsdf_status rtsdf_get_bvh_builder(rtsdf_t ctx, int32_t* builder);

/* Copies the binary topology of the last build to host memory (for checks
 * and tools; synchronises the context's stream).  children: int32
 * [nt - 1][2] (left, right) per node, a child >= 0 is a node, < 0 is
 * ~(leaf position); leaf_tri: int32 [nt], the triangle of each leaf
 * position; root: the root node (-1 when nt < 2).  Any pointer may be NULL
 * to skip that output.  RTSDF_E_STATE without a build. */
rtsdf_status rtsdf_get_bvh_topology(rtsdf_t ctx, int32_t* children, int32_t* leaf_tri, int32_t* root);

/* Sec. 2.1: conservative voxelization.  A coarse voxel is a seed iff some
 * closed triangle meets the closed voxel cube (vertices quantised to 1/256
 * voxel, exact integer separating-axis test). */
rtsdf_status rtsdf_voxelize(rtsdf_t ctx);

/* Sec. 2.1: 3D jump flooding with steps 2^(ceil(log2 N) - 1), ..., 1; each
 * pass takes, per voxel, the nearest seed among the 27 voxels v + {-k,0,k}^3
 * of the previous pass (ties: smaller linear seed index), and the last pass
 * writes the coarse SDF c = h_c sqrt(D2) - beta h_c (fp32). */
rtsdf_status rtsdf_jfa(rtsdf_t ctx);

/* Sec. 2.2 / Eq. 1 for frame `frame`: fine texels whose parent coarse voxel
 * has c <= d_vox * h_c are traced with rays_per_texel (a power of two,
 * 1..1024) random directions from Philox-4x32-10 keyed by (texel, frame,
 * ray); the smallest closest-hit distance r_t updates the accumulator
 * u_t = min(alpha u_{t-1} + (1 - alpha) c_t, r_t) and the front/back hit
 * counts; f_t = +-u_t (minus when back hits outnumber front hits), or c_t
 * while no ray has hit.  Texels with c > d_vox * h_c get f_t = c_t and
 * restart their accumulation.  Requires rtsdf_jfa and rtsdf_build_bvh. */
rtsdf_status rtsdf_trace(rtsdf_t ctx, float d_vox, int32_t rays_per_texel, int32_t frame);

/* Sign statistic of the fine SDF.
 * RTSDF_SIGN_VOTE (default, Sec. 2.2): a texel is negative when its rays'
 *   back-face hits outnumber its front-face hits, counted over frames.
 * RTSDF_SIGN_NEAREST (a variant, not in the paper): a texel takes the face of
 *   the nearest hit found so far (on equal distances a front hit wins), so
 *   no ray needs to look beyond the texel's accumulated distance u: each ray
 *   starts with u as its best hit and culls everything farther.  The
 *   distances u are those of the vote mode (the same rays, the same minimum);
 *   only the sign statistic differs.  In this mode the counts grid holds the
 *   face bit (1 = back) instead of the hit counts.
 * Changing the mode restarts the accumulation (u = +inf, counts 0, f 0);
 * saved states record their mode and rtsdf_load_state adopts it.
 * RTSDF_E_ARG for an unknown mode. */
typedef enum { RTSDF_SIGN_VOTE = 0, RTSDF_SIGN_NEAREST = 1 } rtsdf_sign_mode;
rtsdf_status rtsdf_set_sign_mode(rtsdf_t ctx, int32_t mode);
rtsdf_status rtsdf_get_sign_mode(rtsdf_t ctx, int32_t* mode);

/* Sec. 2.3: soft-shadow visibility.  sdf: float32 [(2N)^3] device grid
 * (NULL = the context's fine SDF).  pos, nrm: float32 [npix, 3] device
 * shading points and unit normals.  light: direction towards the light
 * (host, normalised internally).  Per point the march starts at
 * pos + 2 eps nrm, samples the trilinear SDF, stops with visibility 0 when
 * h < eps, and otherwise returns clamp(min_i k dd_i / (t_i - y_i), 0, 1) over
 * at most `steps` samples (the Aaltonen penumbra estimate), stepping
 * min(h, step_max).  eps = eps_vox h_f, step_max = step_max_vox h_f.
 * vis: float32 [npix] device output.  steps in [1, 256]. */
rtsdf_status rtsdf_shadow(rtsdf_t ctx, const float* sdf, const float* pos, const float* nrm,
                          int64_t npix, const float light[3], float k, int32_t steps,
                          float step_max_vox, float eps_vox, float* vis);

/* Sec. 2.3: rtsdf_shadow with each ray origin jittered toward the light
 * (the paper jitters the origin to break the pattern of constant step sizes
 * and steadies the noise with temporal anti-aliasing, see
 * rtsdf_taa_resolve).  The origin moves by xi x jitter_vox h_f along the
 * light direction, with xi in [0, 1) from Philox-4x32-10 keyed by the
 * context seed and counted by (point index, frame); jitter_vox = 0 gives
 * exactly rtsdf_shadow.  jitter_vox >= 0 and frame >= 0, else RTSDF_E_ARG;
 * the other arguments as rtsdf_shadow.  Counted in the shadow stage. */
rtsdf_status rtsdf_shadow_jittered(rtsdf_t ctx, const float* sdf, const float* pos, const float* nrm,
                                   int64_t npix, const float light[3], float k, int32_t steps,
                                   float step_max_vox, float eps_vox, float jitter_vox, int32_t frame,
                                   float* vis);

/* Sec. 3 (future work in the paper): thin-surface fallback.  The march can
 * step through a surface thinner than its epsilon and leave holes in the
 * umbra; the paper proposes shadow mapping in those regions.  Here: an
 * exact occlusion test of the ray from the march's origin
 * fmaf(nrm, 2 eps_vox h_f, pos) (fp32) along the unit light direction
 * against the context's BVH (the tracer's box and ray/triangle tests; any
 * hit at t >= 0 decides).  Blocked points get vis = 0 in place (vis: float32
 * [npix] device, typically rtsdf_shadow's output; the others keep their
 * value), and blocked (uint8 [npix] device, optional) receives 1 / 0.  The
 * exact test only lowers visibility where the SDF missed an occluder: a
 * thick occluder already stops the march (h < eps).  vis or blocked may be
 * NULL, not both (RTSDF_E_ARG); eps_vox > 0 and a non-zero light as for
 * rtsdf_shadow.  Needs a current BVH (RTSDF_E_STATE after moving objects
 * until rtsdf_build_bvh).  Counted in the shadow stage. */
rtsdf_status rtsdf_shadow_fallback(rtsdf_t ctx, const float* pos, const float* nrm, int64_t npix,
                                   const float light[3], float eps_vox, float* vis, uint8_t* blocked);

/* Sec. 2.3: temporal anti-aliasing of a visibility image for a static view.
 * cur: float32 [height x width] device, this frame (row-major); hist:
 * float32 [height x width] device, the resolved history, updated in place:
 * hist = hc + blend (cur - hc), where hc is hist clamped to the min / max of
 * cur's 3x3 neighbourhood (clamped at the border).  blend in (0, 1]
 * (1 = take cur, e.g. for the first frame).  cur and hist must not overlap;
 * a moving view reprojects hist before the call.  RTSDF_E_ARG on bad
 * sizes, blend or overlapping buffers; an empty image is a no-op. */
rtsdf_status rtsdf_taa_resolve(rtsdf_t ctx, const float* cur, float* hist, int32_t width, int32_t height,
                               float blend);

/* Reverse-mode derivative of rtsdf_shadow (the march is recomputed, not
 * stored).  dvis: float32 [npix] dLoss/dvis.  Accumulates (+=) dLoss/dsdf
 * into dsdf (float32 [(2N)^3], caller-zeroed) and dLoss/dlight into
 * dlight (float32 [3] device, w.r.t. the unnormalised light vector). */
rtsdf_status rtsdf_shadow_backward(rtsdf_t ctx, const float* sdf, const float* pos,
                                   const float* nrm, int64_t npix, const float light[3], float k,
                                   int32_t steps, float step_max_vox, float eps_vox,
                                   const float* dvis, float* dsdf, float* dlight);

/* Jump flooding into caller buffers with no device allocation at all.
 * (Not a step of the paper: an alternative entry point to rtsdf_jfa.)
 * For hosts that cannot call cudaMalloc -- a plug-in running inside another
 * application's memory budget, or a frame loop that bans allocations after
 * start-up because allocating can synchronise the device.  The result equals
 * rtsdf_jfa's: seeds_in is a voxelized seed grid (packed as in rtsdf_grids,
 * 0xFFFFFFFF = no seed), seeds_out receives the nearest seed of every voxel
 * and coarse_out the coarse SDF (h_c = extent / n, beta in coarse voxels);
 * all three are caller-owned device buffers of n^3 elements that must not
 * overlap.  The only scratch is a fixed 8 MiB array inside the library
 * (n <= 128; larger n returns RTSDF_E_ARG), which every GPU that loads the
 * library keeps until the process exits.  The first call in each CUDA
 * context (normally once per device) does a one-time set-up: it looks up
 * that array's device address in the current context and remembers it for
 * that context; make this first call before any stream capture starts.  A
 * context created later (another context on the device, or the primary
 * context again after cudaDeviceReset) gets its own lookup.  All calls share
 * the array, which keeps the last call's contents: two calls that overlap
 * on the GPU (e.g. on different streams) race and both results are
 * undefined.  Work is enqueued on `stream` (NULL = legacy default stream).
 * RTSDF_E_CUDA means the set-up or one of this call's own launches failed;
 * the status is taken from those calls alone, so an error left pending by
 * an unrelated earlier launch is neither returned nor cleared. */
rtsdf_status rtsdf_jfa_noalloc(const uint32_t* seeds_in, uint32_t* seeds_out, float* coarse_out,
                               int32_t n, float extent, float beta_vox, void* stream);

/* ------------------------------------------------------------------------
 * Batched form: many independent scenes (each its own context: grid size,
 * mesh, BVH) updated together.  rtsdf_batch_frame runs the whole per-frame
 * pipeline of Sec. 2.1-2.2 (voxelize, jump flood, mask, trace, Eq. 1) for
 * every scene in one persistent cooperative kernel launch, replayed from a
 * CUDA graph; with split_trace = 1 that launch stops after the mask and the
 * trace and the Eq. 1 finalize of every scene follow as two launches of
 * their own in the same graph.  Each scene's result equals a plain
 * per-scene frame (same kernels' arithmetic, same rays).  Scenes must be
 * static within the batch (no pending rtsdf_move_objects).
 * ------------------------------------------------------------------------ */
typedef struct rtsdf_batch* rtsdf_batch_t;

typedef struct {
    int32_t blocks_per_sm;  /* persistent blocks per SM (0 = occupancy maximum) */
    int32_t refill_min;     /* tracer: refill a warp once this many lanes are idle (1..32) */
    int32_t ray_chunk;      /* tracer: rays a warp takes from the global counter at a time */
    int32_t use_graph;      /* replay the frame from a CUDA graph (1) or launch directly (0) */
    int32_t barrier_spins;  /* polls before a grid-barrier wait gives up with RTSDF_E_TIMEOUT
                               (0 = default, about ten seconds) */
    int32_t leaf_min;       /* tracer: run the leaf phase once this many lanes hold a parked leaf */
    int32_t split_trace;    /* 0: one persistent launch runs every stage; 1: that launch runs the
                               pipeline up to the mask, and the trace and the Eq. 1 finalize follow
                               as two launches of their own in the same frame (and graph), the
                               trace at the per-scene tracer's occupancy; results are identical */
} rtsdf_batch_tuning;

typedef struct {
    int32_t n_scenes;
    int32_t grid;           /* blocks of the persistent launch */
    int32_t graph;          /* 1 when frames replay a captured graph */
    int64_t frames, launches;
    float last_frame_ms;    /* device time of the last frame (CUDA events) */
    /* stage times of the last frame, ms (global timer read at the stage
       barriers; with split_trace, trace runs from the end of the pipeline
       launch to the start of the finalize launch): clear, voxelize, large
       triangles, jump flood, mask, trace, finalize */
    float stage_ms[7];
} rtsdf_batch_info;

/* Creates n scene contexts (1 <= n <= 256) with the given configs.  All
 * scenes share cfgs[0].stream; when it is NULL the batch creates its own
 * non-blocking stream (graph capture cannot use the legacy default stream).
 * Meshes are uploaded and BVHs built per scene through the plain API on the
 * contexts returned by rtsdf_batch_context. */
rtsdf_status rtsdf_batch_create(const rtsdf_config* cfgs, int32_t n, rtsdf_batch_t* out);
rtsdf_status rtsdf_batch_destroy(rtsdf_batch_t batch);
/* Borrowed context of scene i (owned by the batch). */
rtsdf_status rtsdf_batch_context(rtsdf_batch_t batch, int32_t i, rtsdf_t* out);
/* One frame for all scenes (arguments as rtsdf_trace).  Returns
 * RTSDF_E_STATE when a scene lacks a mesh or a current BVH. */
rtsdf_status rtsdf_batch_frame(rtsdf_batch_t batch, float d_vox, int32_t rays_per_texel, int32_t frame);
/* Waits for the batch stream; returns RTSDF_E_TIMEOUT when a bounded
 * grid-barrier wait expired, else the first device error of any scene. */
rtsdf_status rtsdf_batch_sync(rtsdf_batch_t batch);
rtsdf_status rtsdf_batch_set_tuning(rtsdf_batch_t batch, const rtsdf_batch_tuning* t);
rtsdf_status rtsdf_batch_get_tuning(rtsdf_batch_t batch, rtsdf_batch_tuning* t);
rtsdf_status rtsdf_batch_stats(rtsdf_batch_t batch, rtsdf_batch_info* out);

/* Launch parameters of the per-scene path (picked by rtsdf_autotune). */
typedef struct {
    int32_t jfa_tile;            /* jump-flood block tile: 0 = 32x8, 1 = 64x4, 2 = 128x2, 3 = 32x4 voxels,
                                    4 = 32x4 threads flooding 4 voxels each along z (shared z-slices) */
    int32_t trace_blocks_per_sm; /* persistent tracer blocks per SM (0 = occupancy maximum) */
    int32_t refill_min;          /* tracer: refill a warp once this many lanes are idle (1..32) */
    int32_t ray_chunk;           /* tracer: rays a warp takes from the global counter at a time */
    int32_t leaf_min;            /* tracer: run the leaf phase once this many lanes hold a parked leaf (1..32) */
} rtsdf_tuning;

rtsdf_status rtsdf_set_tuning(rtsdf_t ctx, const rtsdf_tuning* t);
rtsdf_status rtsdf_get_tuning(rtsdf_t ctx, rtsdf_tuning* t);

/* Autotuner of the per-scene path: times candidate tunings (CUDA events) on
 * the context's current scene -- jump-flood tiles on rtsdf_jfa, then the
 * tracer's blocks per SM, refill threshold and ray chunk on rtsdf_trace(
 * d_vox, rays, frame) -- keeps the fastest and returns it in best.  The
 * temporal state is saved before and restored after, so the accumulated
 * fine SDF is unchanged.  Results are cached per (device, coarse_n,
 * log2 triangles); use_cache != 0 returns a cached entry without timing.
 * Requires a mesh and a current BVH; synchronises; allocates a temporary
 * copy of the fine grids. */
rtsdf_status rtsdf_autotune(rtsdf_t ctx, float d_vox, int32_t rays_per_texel, int32_t frame, int32_t use_cache,
                            rtsdf_tuning* best);

/* Autotuner of the batched form: blocks per SM, refill threshold and ray
 * chunk of the persistent launch, timed on rtsdf_batch_frame with every
 * scene's temporal state saved and restored.  Cached per (device, scenes,
 * log2 voxels, log2 triangles). */
rtsdf_status rtsdf_batch_autotune(rtsdf_batch_t batch, float d_vox, int32_t rays_per_texel, int32_t frame,
                                  int32_t use_cache, rtsdf_batch_tuning* best);

/* Borrowed device views of the grids (no synchronisation). */
rtsdf_status rtsdf_get_grids(rtsdf_t ctx, rtsdf_grids* out);

/* Number of masked coarse voxels of the last rtsdf_trace (synchronises). */
rtsdf_status rtsdf_get_masked_count(rtsdf_t ctx, int64_t* n_masked_coarse);

/* Statistics (synchronises; resets the per-stage sums and the counters). */
rtsdf_status rtsdf_get_stats(rtsdf_t ctx, rtsdf_stats* out);

/* Per-stage event timing on / off (off by default). */
rtsdf_status rtsdf_set_profiling(rtsdf_t ctx, int on);

/* Tracer work counters on / off (off by default; adds atomics to the tracer,
   so timed runs leave it off). */
rtsdf_status rtsdf_set_counting(rtsdf_t ctx, int on);

/* Checkpoint of the temporal state (accumulator, counts, fine SDF): bytes
 * needed / copy to a host buffer (synchronises) / restore.  Because ray
 * directions depend only on (seed, texel, frame, ray), a restored context
 * continues bit-identically. */
rtsdf_status rtsdf_state_size(rtsdf_t ctx, size_t* bytes);
rtsdf_status rtsdf_save_state(rtsdf_t ctx, void* host_buf, size_t bytes);
rtsdf_status rtsdf_load_state(rtsdf_t ctx, const void* host_buf, size_t bytes);

/* Waits for the context's stream and returns (then clears) any error
 * recorded by device code; RTSDF_E_CUDA on a CUDA error. */
rtsdf_status rtsdf_sync(rtsdf_t ctx);

/* Static description of a status code. */
const char* rtsdf_status_str(rtsdf_status s);

/* Library version, "major.minor.patch". */
const char* rtsdf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RTSDF_H */
