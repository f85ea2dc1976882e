/*
 * mars.h -- C ABI of the GB300 MARS path tracer.
 *
 * MARS (Meyer, Rath, Yazici, Slusallek, "MARS: Multi-sample Allocation through
 * Russian roulette and Splitting", SIGGRAPH Asia 2024) renders an image by
 * iterating a fixed-point scheme: every iteration traces paths in which each
 * vertex draws a real-valued number of samples beta_t per technique t (BSDF
 * sampling, next-event estimation, guided sampling), rounds them with
 * low-discrepancy stochastic rounding (Alg. 1), combines the samples with the
 * multi-sample balance heuristic (Sec. 3.1, "Secondary estimator") and records
 * per-cell moment and cost estimates (Sec. 4.1, "Local estimates").  The update
 * step turns those estimates, the image variance V_I and the image cost C_I
 * into the next iteration's counts (Eq. "optimalBeta" in the spatial form of
 * Sec. 3.1, "Optimization").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All calls return a mars_status.  Nothing is thrown across the ABI.  The
 *   message of the last failure on the calling thread is available through
 *   mars_last_error_string().
 * - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 * - Descriptors and host arrays are owned by the caller and copied during the
 *   call.  Objects (mars_scene, mars_cache, mars_server) are owned by the
 *   library until the matching *_destroy.
 * - Objects live on the CUDA device that was current when they were created;
 *   every call switches to that device for its duration.
 * - After MARS_ERR_CUDA an object is poisoned: every later call on it fails
 *   with MARS_ERR_CUDA and only *_destroy is meaningful.
 * - The library never falls back to the CPU.
 */
#ifndef MARS_H
#define MARS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MARS_OK = 0,
  MARS_ERR_INVALID_ARG = 1, /* a pointer, size or enum is out of range */
  MARS_ERR_OOM = 2,         /* device memory, or a single pixel's path tree exceeds the queue arena */
  MARS_ERR_CUDA = 3,        /* a CUDA runtime call failed; the object is poisoned */
  MARS_ERR_TIMEOUT = 4,     /* a bounded wait ran out */
  MARS_ERR_BUSY = 5,        /* the server has no free slot for the request right now */
  MARS_ERR_NOT_FOUND = 6    /* unknown job id */
} mars_status;

typedef struct mars_scene mars_scene;
typedef struct mars_cache mars_cache;
typedef struct mars_server mars_server;

/* technique bits and slots; slots are the order Alg. 1 rounds in.
 * MARS_TECH_LIGHT: connections to light subpaths, the third technique of the
 * bidirectional application (Sec. 5); it takes slot 2 and excludes
 * MARS_TECH_GUIDED.  A light connection sample at camera vertex x_i traces one
 * light subpath of its own (light and point chosen as for NEE, cosine
 * emission, BSDF sampling and throughput-based Russian roulette at every
 * surface vertex, at most MARS_LIGHT_MAX surface vertices and D - 1 - i) and
 * connects x_i to each of its surface vertices; it is drawn at vertices of
 * depth <= D - 2.  With it, every contribution is weighted by the
 * budget-aware balance heuristic over all strategies of its full path (camera
 * path, NEE at the last vertex, light connection at any earlier one), and the
 * local outlier clamp is off (Sec. 5.1). */
#define MARS_TECH_BSDF 1
#define MARS_TECH_NEE 2
#define MARS_TECH_GUIDED 4
#define MARS_TECH_LIGHT 8
#define MARS_SLOT_BSDF 0
#define MARS_SLOT_NEE 1
#define MARS_SLOT_GUIDED 2
#define MARS_SLOT_LIGHT 2
#define MARS_NUM_SLOTS 3
#define MARS_LIGHT_MAX 5      /* surface vertices of a light subpath (6 vertices with the light's) */
#define MARS_NUM_STATS 8      /* n, sum v (rgb), sum v^2 (rgb), sum cost */
#define MARS_GUIDE_BINS 256   /* 16 (cos theta) x 16 (phi) equal-area bins */
#define MARS_MAX_DEPTH 16

typedef enum { MARS_MODE_WARMUP = 0, MARS_MODE_MARS = 1, MARS_MODE_FIXED = 2 } mars_mode;
typedef enum { MARS_WEIGHTS_AWARE = 0, MARS_WEIGHTS_UNAWARE = 1 } mars_weights;

/* Scene description (host memory, copied by mars_scene_create).
 * quads [n_quads][9]: corner p0, edge e1, edge e2; a quad whose material emits
 *   is an area light, emitting on the side of normalize(e1 x e2).
 * spheres [n_spheres][4]: centre, radius.   tris [n_tris][9]: v0, v1, v2.
 * *_mat: material index per primitive.  Only quads may use emitting materials.
 * materials [n_materials][8]: type (0 Lambert, 1 GGX), colour rgb (Lambertian
 *   albedo, or GGX Fresnel F0), GGX roughness alpha, emitted radiance rgb.
 * camera: pinhole origin, look-at point, up vector, vertical FOV in degrees;
 *   width x height pixels, one box-filtered sample per pixel per iteration.
 * bvh: the hierarchy the closest-hit and shadow queries traverse (results do
 *   not depend on it): MARS_BVH_SAH (0) a top-down build on the host with the
 *   surface-area heuristic; MARS_BVH_LBVH a linear BVH built on the device
 *   (Morton codes, Karras hierarchy).  reserved: 0. */
#define MARS_BVH_SAH 0
#define MARS_BVH_LBVH 1
typedef struct {
  int32_t n_quads, n_spheres, n_tris, n_materials;
  const double* quads;
  const int32_t* quad_mat;
  const double* spheres;
  const int32_t* sphere_mat;
  const double* tris;
  const int32_t* tri_mat;
  const double* materials;
  double camera[10];
  int32_t width, height;
  int32_t bvh, reserved;
} mars_scene_desc;

/* Statistics cache and iteration state of one render job.
 * grid_n: uniform N^3 grid over the scene bounds (Sec. 4.1 stores the local
 *   estimates in a spatial data structure; a uniform grid stands in for it).
 * techniques: MARS_TECH_* bits; BSDF is required.
 * max_depth: maximum number of path segments D (1..MARS_MAX_DEPTH); vertices
 *   x_1..x_{D-1} run the secondary estimator.
 * flags: MARS_CACHE_FP32_STATISTICS: accumulate the local statistics, run the
 *   count update and reduce V_I and C_I in float32 instead of float64 (the
 *   float32-only variant of the precision study; default float64).
 *   MARS_CACHE_OCTREE: an adaptive octree over the scene box instead of the
 *   uniform grid (the EARS octree of Sec. 5.1): it starts as the grid (grid_n
 *   a power of two, cells numbered as in the grid) and after every
 *   mars_update_counts splits, in cell order, each leaf that received at least
 *   split_samples samples (all techniques) in the iteration into 8 children,
 *   down to 1024 cells per axis and while the leaves number at most
 *   max_leaves; children inherit the counts and the guide distribution.
 *   MARS_CACHE_NO_GRAPHS: launch every kernel of an iteration directly.  By
 *   default an iteration whose pixel tiles fit the arena at the first attempt,
 *   is not profiled and runs on a stream other than the legacy default stream
 *   (which cannot be captured) is recorded once as a CUDA graph and replayed;
 *   the graph is recorded again when the output buffer, update_estimate, the
 *   image-statistics options, the tile count or the launch shape change.
 *   MARS_CACHE_ONE_LANE: one tile lane.  By default the pixels are split into
 *   tiles dealt to two lanes, each with half the arena, its own streams and
 *   counters, rendered concurrently (their wave kernels fill each other's idle
 *   SMs).  Results are the same either way (statistics up to the order of
 *   float64 atomics).
 * max_leaves, split_samples: octree only (0: 65536 leaves, 4096 samples).
 * arena_capacity: rays held by the per-iteration queue arena summed over all
 *   depths (0 = 3 x pixels x max_depth, at least 2^20); as many NEE shadow-ray
 *   slots, and with light connections as many connection-sample and light-vertex
 *   slots.  An iteration whose path trees do not fit is rendered in pixel tiles
 *   (results do not depend on it). */
#define MARS_CACHE_FP32_STATISTICS 1
#define MARS_CACHE_OCTREE 2
#define MARS_CACHE_NO_GRAPHS 4
#define MARS_CACHE_ONE_LANE 8
#define MARS_OCTREE_MAX_LEVEL 10
typedef struct {
  int32_t grid_n;
  int32_t techniques;
  int32_t max_depth;
  int32_t flags;
  uint64_t arena_capacity;
  int32_t max_leaves;
  float split_samples;
} mars_cache_desc;

/* Per-iteration parameters.
 * seed, job: Philox key.  iteration: fixed-point iteration index (< 65536);
 *   it keys the random numbers, so re-rendering an iteration reproduces it.
 * mode: WARMUP and FIXED draw one sample per technique (beta = 1); MARS reads
 *   the counts from the cache (Sec. 3.1 "Optimization").
 * weights: budget-aware (default) or budget-unaware balance heuristic.
 * clamp_lo/hi: count clamp (0.05, 20 in Sec. 4.1); clamp_hi <= 30.
 * outlier: multiple of the pixel estimate that bounds a sample's contribution
 *   to the variance estimates (50 in Sec. 4.1), not to the image.
 * collect: accumulate local statistics and guide deposits.
 * image_on_host: image_rgb is host memory (the call copies the image back).
 * update_estimate: after rendering, add the image to the running mean and
 *   recompute the pixel estimate, V_I and C_I (needed before mars_update_counts).
 * profile: time every kernel launch with CUDA events on `stream`; the device
 *   time per stage is returned in mars_iter_stats.
 * vi_drop_brightest: K in 0..MARS_MAX_DROP_BRIGHTEST.  K > 0 replaces the
 *   outlier clamp of V_I by the rejection of the bidirectional application
 *   (Sec. 5.1 "Implementation"): the K pixels of highest luminance of the
 *   iteration's image (0.2126 R + 0.7152 G + 0.0722 B in float32; ties to the
 *   lower pixel index) leave the V_I mean, the others enter unclamped.
 * combine: progressive combination of Sec. 5.1 (the inverse-variance weighted
 *   combination of iterations): 1 adds this iteration's image with weight
 *   1 / max(V_I, 1e-12) to the cache's combined image, 2 starts a new
 *   combination with it; needs update_estimate.  Read it with
 *   mars_cache_combined_image.
 * Pixel ranges (px_begin < px_end <= pixels): only the camera paths of those
 *   pixels are traced.  Every camera path is independent within an iteration
 *   (Sec. 3.1 "Random walks"), and its random numbers depend on its pixel index
 *   only, so a frame split into ranges rendered by several caches (one per GPU)
 *   gives, range by range, the pixels of the whole-frame render, and the
 *   statistics, rays, vertices and beta sums of the ranges add up to the whole
 *   frame's (up to the order of the float64 sums).  This is the partitioning of
 *   a multi-GPU job: each rank renders its range, the float64 statistics and
 *   the counters are summed across ranks, and the update runs on the sum.  A
 *   range needs update_estimate = 0 and combine = 0 (the image statistics
 *   filter across the whole image); image_rgb still spans the whole frame and
 *   only the range's pixels are written. */
#define MARS_MAX_DROP_BRIGHTEST 16
typedef struct {
  uint32_t seed, job, iteration;
  int32_t mode;
  int32_t weights;
  float clamp_lo, clamp_hi, outlier;
  int32_t collect;
  int32_t image_on_host;
  int32_t update_estimate;
  int32_t profile;         /* record CUDA events around every kernel (stage times in mars_iter_stats) */
  float max_multiplicity;  /* path multiplicity cap M (0 = none, the paper's rule): every budget is
                              further limited to max(clamp_lo, M / P), P = the product of the budgets
                              that drew the path so far, so one camera sample spawns at most M
                              vertices per depth in expectation; any budget field stays unbiased */
  int32_t vi_drop_brightest;  /* K brightest pixels left out of V_I (0: the outlier clamp) */
  int32_t combine;            /* 0 none, 1 add to, 2 restart the inverse-variance combination */
  int32_t px_begin, px_end;   /* pixel range [px_begin, px_end) in row-major order (both 0: every
                                 pixel); see "Pixel ranges" below */
} mars_iter_params;

/* What one iteration did (host memory, filled by mars_render_iteration). */
typedef struct {
  double VI;                  /* image relative variance (Sec. 4.1, "Image estimates") */
  double CI;                  /* rays per pixel (cost units, Sec. 4.1) */
  uint64_t rays;              /* camera rays + every drawn technique sample */
  uint64_t vertices;          /* closest-hit queries (camera and extension rays traced) */
  uint64_t estimator_vertices;/* vertices that ran the secondary estimator */
  double mean_beta[3];        /* mean beta per technique slot over estimator vertices */
  uint32_t tiles;             /* pixel tiles used (1 unless the arena overflowed) */
  uint32_t retries;           /* tiles re-rendered after an overflow */
  uint64_t arena_demand;      /* rays the largest tile needed */
  uint32_t launches;          /* kernels this call launched */
  uint32_t wave_launches;     /* launches of each per-wave kernel (depth waves x tiles) */
  /* device time per kernel kind, summed over waves and tiles (profile = 1) */
  double trace_ms, shade_ms, shadow_ms, reverse_ms, image_ms;
  uint64_t wave_entries;      /* rays held in the depth waves (traced or not), all tiles */
  uint64_t shadow_entries;    /* NEE shadow-ray slots, all tiles */
  uint64_t shadow_traced;     /* NEE shadow rays traced (samples of nonzero value), all tiles */
  float wave_ms[4][16];       /* profile = 1: device ms of trace, shade, shadow, reverse per depth wave d (index d - 1) */
  uint64_t wave_rays[16];     /* rays held by depth wave d (index d - 1), all tiles */
  uint64_t trace_work[2][4];  /* closest-hit [0] and shadow [1] traversal: BVH node visits
                                 (two box tests each), quad, sphere and triangle tests */
  uint32_t check_flags;       /* MARS_CHECK_* bits of the index checks that failed (always 0
                                 in the regular library; see below) */
  uint32_t reserved;
  /* light connections (MARS_TECH_LIGHT): light-subpath closest-hit queries
     (included in `vertices`), connection shadow rays traced, light connection
     samples drawn, and (profile = 1) the device time of their kernels (the
     light-subpath and connection kernels of every wave) */
  uint64_t light_rays, connection_rays, light_samples;
  double light_ms;
} mars_iter_stats;

/* Index checks of the checked library (libmars_checked.so, the same sources
 * built with MARS_CHECKED): kernels test every arena slot, cell, pixel, BVH node,
 * primitive, material, light and guide-bin index they compute against the
 * buffer it addresses, skip an access that fails, and report the kind here
 * (compute-sanitizer is unavailable; no check traps or faults). */
#define MARS_CHECK_ARENA 1u
#define MARS_CHECK_SHADOW 2u
#define MARS_CHECK_CELL 4u
#define MARS_CHECK_PIXEL 8u
#define MARS_CHECK_PRIM 16u
#define MARS_CHECK_NODE 32u
#define MARS_CHECK_LIGHT 64u
#define MARS_CHECK_BIN 128u
#define MARS_CHECK_MATERIAL 256u

/* Host copy of a cache's state (checkpoint / teacher forcing).  Any pointer
 * may be NULL to skip that field.  Layouts:
 * q_rr, q_s [cells][3][3]: count factors per (cell, technique slot, channel):
 *   q = sqrt(C_I / C_t * M_t / V_I) with M_t the second moment (RR) or the
 *   variance (S) of the technique's samples in the cell.
 * valid [cells][3]: 0 -> the vertex uses beta = 1 for that technique.
 * stats [cells][3][8]: n, sum v (rgb), sum v^2 (rgb), sum cost (float64).
 * guide_hist [cells][256]: accumulated guide deposits.
 * guide_cdf [cells][256]: inclusive CDF of the guided technique per cell.
 * pixel_estimate [pixels][3], run_sum [pixels][3]: float32.
 * Octree caches: cells = max_leaves (only the first oct_n_leaves are in use);
 * oct_nodes [oct_n_nodes] int32: node >= 0 is the index of its first of 8
 * children (octant = x | y << 1 | z << 2), < 0 a leaf ~cell; oct_leaf_level
 * [oct_n_leaves] int32.  set_state takes a tree when oct_nodes is non-NULL. */
typedef struct {
  float* q_rr;
  float* q_s;
  uint8_t* valid;
  double* stats;
  float* guide_hist;
  float* guide_cdf;
  float* pixel_estimate;
  float* run_sum;
  int32_t n_iterations;   /* iterations summed in run_sum */
  int32_t has_estimate;   /* pixel_estimate is meaningful */
  double VI, CI;          /* inputs of the next mars_update_counts: the means over the
                             image_iterations iterations rendered with update_estimate
                             since the last update (0 when there were none) */
  int32_t* oct_nodes;
  int32_t* oct_leaf_level;
  int32_t oct_n_nodes, oct_n_leaves;
  float* pixel_rays;      /* get_state only: [pixels] rays of each pixel's path tree in the last
                             rendered iteration (its camera ray and every sample drawn below it) */
  int32_t image_iterations; /* iterations averaged into VI and CI; set_state takes 0 as one
                               when VI or CI is non-zero */
} mars_cache_state;

typedef struct {
  int64_t n_cells, n_pixels;
  int32_t grid_n, techniques, max_depth, n_prims;
  uint64_t arena_capacity;
  uint64_t device_bytes;
  int32_t device;
  int32_t n_lights;
  int32_t oct_n_nodes, oct_n_leaves;  /* octree caches: current tree size (0 for a grid) */
  int32_t oct_cap_nodes;              /* octree caches: node capacity (state buffers) */
  int32_t graph_captures;             /* iteration graphs recorded so far */
} mars_cache_info;

/* ---- scene ------------------------------------------------------------
 * Copies the description to the device, builds the closest-hit hierarchy
 * selected by desc->bvh -- by default (MARS_BVH_SAH) a top-down surface-area
 * heuristic build on the host CPU (binned above 64 primitives, exact sweeps
 * below; about 0.1 s for 131k triangles, 0.4 s for 524k), with MARS_BVH_LBVH a
 * linear BVH built on the device (Morton codes, sort, Karras hierarchy,
 * bottom-up bounds); either is validated on the host and collapsed into the
 * 4-wide hierarchy of the shadow rays -- and the light-selection table
 * (probability proportional to area x mean radiance).  Results do not depend
 * on the hierarchy.  Synchronises `stream` before returning.  Errors: INVALID_ARG (no primitives, bad sizes,
 * material index out of range, emitting sphere/triangle), OOM, CUDA. */
mars_status mars_scene_create(const mars_scene_desc* desc, void* stream, mars_scene** out);
mars_status mars_scene_destroy(mars_scene* scene);

/* ---- cache --------------------------------------------------------------
 * Allocates the statistics cache, count fields (all invalid: beta = 1), guide
 * (uniform), image accumulators and the queue arena for `scene`, which must
 * outlive the cache.  Synchronises `stream`.  Errors: INVALID_ARG, OOM, CUDA.
 * Scene and cache memory comes from the device's stream-ordered memory pool,
 * which keeps released memory for the next object; *_destroy waits for the
 * stream of the object's last call and releases the memory there. */
mars_status mars_cache_create(const mars_scene* scene, const mars_cache_desc* desc, void* stream,
                              mars_cache** out);
mars_status mars_cache_destroy(mars_cache* cache);
mars_status mars_cache_info_get(const mars_cache* cache, mars_cache_info* info);

/* ---- one render of a training iteration (Sec. 4.1, "Fixed-point iteration") -
 * Renders one sample per pixel with the wavefront MARS path tracer: camera
 * rays, then per depth wave closest hit, count lookup (T(x)/I_px x q, three
 * cases, clamp), Alg. 1, NEE shadow rays, BSDF/guided child rays compacted
 * into the next wave; then a deepest-first pass that forms every sample's value
 * and cost and scatters the local statistics.  image_rgb [height][width][3]
 * float32 receives the iteration's one-sample image (device memory unless
 * params->image_on_host).  stats_host may be NULL.  Statistics accumulate
 * until mars_update_counts.  The call synchronises `stream` once at the end
 * (twice if the arena overflowed and tiles were re-rendered).
 * Errors: INVALID_ARG (MARS mode without a pixel estimate, clamp_hi > 30,
 * iteration >= 65536), OOM (a single pixel's path tree exceeds the arena), CUDA. */
mars_status mars_render_iteration(mars_cache* cache, const mars_iter_params* params, float* image_rgb,
                                  mars_iter_stats* stats_host, void* stream);

/* ---- fixed-point update (Sec. 3.1 "Optimization"; App. A.3) -----------------
 * Closes one training iteration: every mars_render_iteration since the last
 * update (one or several samples per pixel; the paper's training iterations
 * grow in duration, Sec. 4.1 "Fixed-point iteration" and Sec. 5.1) added its
 * statistics, and each one with update_estimate its V_I and C_I.  One step per
 * (cell, technique): q^RR and q^S per channel from the collected statistics and
 * the means of those V_I and C_I (the paper's V_I averages the squared relative
 * errors over every sample of the iteration, Sec. 4.1 "Image estimates");
 * keeps the previous factors where n < 2 or the cost is 0, and everything when
 * V_I <= 1e-12 (no image statistics ran).  Rebuilds the guided technique's per-cell CDF
 * from the accumulated deposits (P_b = 0.9 h_b / H + 0.1 / 256).  Zeroes the
 * statistics.  Asynchronous on `stream`.  Errors: CUDA. */
mars_status mars_update_counts(mars_cache* cache, void* stream);

/* ---- training schedule (Sec. 4.1 "Fixed-point iteration"; Sec. 5.1) ---------
 * The paper's training iterations grow in duration (the guided application
 * follows the guiding scheme it builds on, whose iterations double; the
 * bidirectional one renders "short iterations that grow in duration").  A job
 * of `iterations` one-sample renders whose first `warmup` are warm-up renders
 * is split into training iterations: each warm-up render is one, then 1, 2, 4,
 * ... renders, the last one taking what is left; an iteration after which
 * fewer renders than its own would remain takes them too (no short last
 * iteration replaces counts learned from a long one).  Returns 1 when render
 * `iteration` (0-based) closes a training iteration, i.e. mars_update_counts
 * follows it, else 0 (also for iteration < 0, iteration >= iterations or
 * warmup < 0).  Host only; no device work. */
int32_t mars_training_step_ends(int32_t iteration, int32_t warmup, int32_t iterations);

/* ---- testing hook (host only; the paper has no counterpart) -------------
 * Exercises the error paths without faulting a GPU.  kind MARS_INJECT_ALLOC:
 * the n-th next device allocation of the library, in any call, fails as if the
 * device were out of memory (the call returns MARS_ERR_OOM and releases what
 * it had allocated).  kind MARS_INJECT_LAUNCH: the n-th next
 * mars_render_iteration or mars_update_counts fails as if a kernel launch had
 * failed (MARS_ERR_CUDA; that cache is poisoned, others are unaffected).
 * n = 0 cancels.  Process-wide countdowns.  Errors: INVALID_ARG. */
#define MARS_INJECT_ALLOC 0
#define MARS_INJECT_LAUNCH 1
mars_status mars_debug_inject_failure(int32_t kind, int32_t n);

/* ---- progressive combination (Sec. 5.1 "Implementation") ----------------
 * The combined image sum_i w_i I_i / sum_i w_i over the iterations rendered
 * with params.combine (w_i = 1 / max(V_I of iteration i, 1e-12)), packed rgb
 * float32 [height][width][3] into host memory image_rgb, and sum_i w_i into
 * *weight_sum (either may be NULL).  Zeros while nothing was combined.
 * Synchronises `stream`.  Errors: INVALID_ARG, OOM (staging buffer), CUDA. */
mars_status mars_cache_combined_image(mars_cache* cache, float* image_rgb, double* weight_sum, void* stream);

/* ---- state transfer (checkpoint / resume, teacher-forced checks) ----------
 * Synchronous copies of the fields whose pointers are non-NULL. */
mars_status mars_cache_get_state(mars_cache* cache, mars_cache_state* state, void* stream);
mars_status mars_cache_set_state(mars_cache* cache, const mars_cache_state* state, void* stream);

/* ---- launch shape and autotuning ---------------------------------------------
 * The four per-wave kernels (closest hit, shading and sampling, NEE shadow
 * rays, deepest-first reverse pass) each run a persistent grid of
 * SMs x blocks_per_sm blocks that strides over its wave in chunks of 32 slots;
 * the launch shape changes their speed, never their results.
 * threads[k]: threads per block of kernel k (0 trace, 1 shade, 2 shadow,
 *   3 reverse), a multiple of 32 in 32..256.
 * blocks_per_sm[k]: 1..64, or 0 = as many blocks as fit on an SM at once
 *   (mars_cache_get_launch reports the resolved count).
 * max_registers[k]: selects a compiled variant of the kernel whose registers
 *   per thread are capped (more resident blocks, possibly some spilling).
 * lanes: concurrent tile lanes an iteration may use, 1 up to the count the
 *   cache was created with (two, or one with MARS_CACHE_ONE_LANE); 0 keeps the
 *   current value in mars_cache_set_launch.
 * lane_min_pixels: the smallest image split over the lanes (default 2^17;
 *   at least 2); 0 keeps the current value.
 * Default: 128 threads, no cap, the occupancy maximum, every depth wave on the
 * same grid.  Errors: INVALID_ARG, CUDA. */
typedef struct {
  int32_t threads[4];
  int32_t blocks_per_sm[4];
  int32_t max_registers[4];  /* register cap of the compiled variant: 0 = the compiler's
                                choice; shade and reverse also 80 or 64, trace and shadow 64 or 40 */
  int32_t lanes;
  int32_t lane_min_pixels;
} mars_launch_config;
mars_status mars_cache_get_launch(const mars_cache* cache, mars_launch_config* out);
mars_status mars_cache_set_launch(mars_cache* cache, const mars_launch_config* config);
/* Picks each wave kernel's launch shape in turn (register-cap variant x threads
 * per block in {64, 128, 256} x blocks per SM in {half, full, twice} the
 * occupancy maximum)
 * by the kernel's device time over `repeats` (1..100) renders of `params`'s
 * iteration, rendered without statistics, guide deposits or image statistics
 * so that the cache's learned state is unchanged; keeps the fastest shape.
 * Then, for a cache with more than one lane and an image of at least 2^14
 * pixels, times whole iterations (as rendered outside profiling: graphs, lanes)
 * with one lane and with all lanes for any image of that size, and keeps the
 * faster.  Writes the result to `chosen` (may be NULL).  Synchronises `stream`
 * after every render.  Errors: INVALID_ARG, and those of mars_render_iteration. */
mars_status mars_cache_autotune(mars_cache* cache, const mars_iter_params* params, int32_t repeats,
                                mars_launch_config* chosen, void* stream);

/* ---- serving ----------------------------------------------------------------
 * A server owns a host scheduler thread that admits render jobs while their
 * estimated device footprint fits `memory_budget_bytes` and fewer than
 * `max_slots` jobs are resident, and runs every admitted job's iterations on
 * its own stream so that jobs overlap on the device. */
typedef struct {
  const mars_scene_desc* scene;
  mars_cache_desc cache;
  uint32_t seed;           /* Philox key of the job: (seed, key) */
  int32_t iterations;      /* one-sample renders of the job; the count update follows
                              the renders that mars_training_step_ends names */
  int32_t warmup;          /* leading renders with beta = 1 */
  uint32_t key;            /* second Philox key word; a job's random numbers depend
                              on (seed, key) only, never on the server's job id */
  double timeout_s;        /* wall-clock limit counted from the job's start (0: none):
                              a job still running past it stops before its next
                              iteration and fails with MARS_ERR_TIMEOUT */
} mars_job_desc;

typedef enum { MARS_JOB_QUEUED = 0, MARS_JOB_RUNNING = 1, MARS_JOB_DONE = 2, MARS_JOB_FAILED = 3 } mars_job_state;

typedef struct {
  int32_t state;           /* mars_job_state */
  int32_t iterations_done;
  int32_t error;           /* mars_status of a failed job */
  int32_t reserved;
  double submit_s, start_s, end_s;   /* wall-clock seconds since server creation */
  double iter_ms_p50, iter_ms_p99;   /* per-iteration latency */
  uint64_t device_bytes;             /* device memory the job was admitted with */
  uint64_t vertices;                 /* path vertices (closest-hit queries) over the done iterations */
} mars_job_status;

mars_status mars_server_create(uint64_t memory_budget_bytes, int32_t max_slots, mars_server** out);
mars_status mars_server_destroy(mars_server* server);
/* Queues a job (the scene description is copied).  Never blocks on the GPU. */
mars_status mars_submit(mars_server* server, const mars_job_desc* job, uint64_t* job_id);
/* Status of a job; when done, image_rgb (host, width*height*3 float32, may be
 * NULL) receives the mean image over its iterations after warm-up. */
mars_status mars_poll(mars_server* server, uint64_t job_id, mars_job_status* out, float* image_rgb);

/* Per-iteration latencies of a job in milliseconds (render + update, host wall
 * clock around the job stream's synchronisation), in iteration order: writes
 * min(capacity, done iterations) values to ms (host) and the number of done
 * iterations to *count.  Errors: INVALID_ARG, NOT_FOUND. */
mars_status mars_job_latencies(mars_server* server, uint64_t job_id, double* ms, int32_t capacity, int32_t* count);
/* ---- image statistics without allocation ------------------------------------
 * The paper has no counterpart to this entry point; it is a library service.
 * Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
 * being captured, allocator-less embedded hosts, or a serving process whose
 * device memory is fully reserved up front.  For them this call computes the
 * same per-iteration image statistics as mars_render_iteration with
 * update_estimate = 1 (running sum, pixel estimate, V_I and C_I) -- for a cache
 * with float64 statistics and vi_drop_brightest = 0: its V_I clamps every
 * sample at `outlier` x the pixel estimate and averages over all pixels, and it
 * has no float32 variant and no brightest-pixel rejection -- directly on
 * caller buffers and allocates nothing: its only scratch is a static device
 * array of the library (256 KB, held by every GPU that loads the library until
 * the process exits), with room for images of at most 8192 rows.
 *   image_rgb    [height][width][3] float32, device: this iteration's image.
 *   run_sum_rgb  [height][width][3] float32, device, in/out: sum over the
 *                n_prev earlier iterations; the image is added to it.
 *   estimate_rgb [height][width][3] float32, device, out: pixel estimate.
 *   vi_ci        2 float64, device, out: V_I and C_I = rays / pixels.
 * Asynchronous on `stream`.  The first call on a device looks up the scratch
 * array's device address (cudaGetSymbolAddress) and must therefore come before
 * any stream capture on that device.  The address is cached for the life of
 * the process: after cudaDeviceReset (or anything else that destroys the
 * device's primary context) this entry point must not be called again on that
 * device.  All calls share the scratch array: calls
 * whose work overlaps on the GPU race and give wrong results; serialise them.
 * Errors: INVALID_ARG (null pointer, height above 8192 rows, bad sizes), CUDA. */
mars_status mars_image_stats_static(const float* image_rgb, float* run_sum_rgb, float* estimate_rgb, int32_t width,
                                    int32_t height, int32_t n_prev, float outlier, double rays, double* vi_ci,
                                    void* stream);

/* ---- diagnostics ------------------------------------------------------------ */
const char* mars_last_error_string(void);
const char* mars_version(void);

#ifdef __cplusplus
}
#endif
#endif
