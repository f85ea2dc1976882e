/*
 * mars_oracle.h -- plain CPU oracle for MARS (Meyer, Rath, Yazici, Slusallek,
 * "MARS: Multi-sample Allocation through Russian roulette and Splitting",
 * SIGGRAPH Asia 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no source with the CUDA path.
 *
 * Everything is float64 except the few quantities that arrive as float32
 * inputs (count factors, pixel estimates, guide CDFs) and the stochastic
 * rounding decision of Alg. 1, which is taken in float32 (the precision the
 * CUDA path takes it in) so that both sides decide integers in the same
 * precision.
 */
#ifndef MARS_ORACLE_H
#define MARS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* technique slots (fixed order BSDF, NEE, guided or light connection; Alg. 1
 * rounds in this order).  Technique bits: 1 BSDF, 2 NEE, 4 guided, 8 light
 * connection (the bidirectional application, Sec. 5); guided and light
 * connection share slot 2 and exclude each other. */
#define ORC_T_BSDF 0
#define ORC_T_NEE 1
#define ORC_T_GUIDED 2
#define ORC_T_LIGHT 2
#define ORC_NT 3
#define ORC_TECH_LIGHT 8
/* surface vertices of a light subpath at most (the light vertex y_0 plus 5:
 * light subpaths of at most 6 vertices) */
#define ORC_LIGHT_MAX 5
/* per (cell, technique) statistics: n, sum v[3], sum v^2[3], sum cost */
#define ORC_NSTAT 8
#define ORC_GUIDE_BINS 256

typedef struct {
  int n_quads, n_spheres, n_tris, n_materials;
  const double* quads;      /* [n_quads][9]  p0, e1, e2 */
  const int32_t* quad_mat;
  const double* spheres;    /* [n_spheres][4] centre, radius */
  const int32_t* sphere_mat;
  const double* tris;       /* [n_tris][9] v0, v1, v2 */
  const int32_t* tri_mat;
  const double* materials;  /* [n_materials][8] type, rgb, alpha, Le rgb */
  double camera[10];        /* origin, look-at, up, vertical fov (degrees) */
  int width, height;
} orc_scene_desc;

typedef enum { ORC_MODE_WARMUP = 0, ORC_MODE_MARS = 1, ORC_MODE_FIXED = 2 } orc_mode;
typedef enum { ORC_WEIGHTS_AWARE = 0, ORC_WEIGHTS_UNAWARE = 1 } orc_weights;

typedef struct {
  int grid_n;           /* statistics grid resolution N (N^3 cells) */
  int techniques;       /* bit 0 BSDF, bit 1 NEE, bit 2 guided */
  int max_depth;        /* D: maximum number of path segments */
  int mode;             /* orc_mode */
  int weights;          /* orc_weights */
  uint32_t seed, job;   /* Philox key */
  uint32_t iteration;   /* fixed-point iteration index (< 65536) */
  double clamp_lo, clamp_hi;  /* count clamp, [0.05, 20] in the paper */
  double outlier;       /* outlier multiple of the pixel estimate (50) */
  int has_estimate;     /* 1 if est[] holds a pixel estimate */
  int collect;          /* 1: accumulate statistics and guide deposits */
  float max_mult;       /* path multiplicity cap M (0: none), see orc_render */
} orc_params;

typedef struct {
  /* inputs */
  const float* q_rr;          /* [cells][3][3] */
  const float* q_s;           /* [cells][3][3] */
  const uint8_t* valid;       /* [cells][3] */
  const float* guide_cdf;     /* [cells][256] inclusive CDF (guided only) */
  const float* est;           /* [pixels][3] pixel estimate */
  const int32_t* oct_nodes;   /* adaptive octree over the scene box (NULL: the uniform grid_n^3 grid);
                                 node >= 0: first of its 8 children, < 0: leaf ~cell */
  /* outputs (accumulated, caller zeroes) */
  double* image;              /* [pixels][3] one-sample pixel estimate (written) */
  double* stats;              /* [cells][3][8] */
  double* hist;               /* [cells][256] guide deposits */
  double* counters;           /* [0] rays (cost units) [1] closest-hit queries (camera and light
                                 paths) [2] estimator vertices [3..5] sum of beta per technique
                                 [6] light-path closest-hit queries [7] connection rays traced */
  double* px_rays;            /* [pixels] rays of each pixel's path tree (written; may be NULL) */
} orc_state;

/* Render pixels [px_begin, px_end) of one iteration depth-first.  Returns 0 on
 * success, a negative value on invalid input. */
int orc_render(const orc_scene_desc* scene, const orc_params* params, orc_state* st,
               int px_begin, int px_end);

/* Image statistics after an iteration: run_sum += img; mean = run_sum / (n_prev+1);
 * est_out = max(3x3 box(mean), 1e-3 * channel mean, 1e-8);
 * returns V_I = mean over pixels and channels of ((min(img, outlier*est) - est)/est)^2. */
double orc_image_stats(int width, int height, const double* img, double* run_sum,
                       int n_prev, double outlier, double* est_out);
/* The same with drop_k > 0: V_I instead leaves out the drop_k brightest pixels
 * (float32 luminance, ties to the lower index) and clamps no sample (the
 * rejection of the bidirectional application, Sec. 5.1).  drop_k = 0: as above. */
double orc_image_stats_k(int width, int height, const double* img, double* run_sum,
                         int n_prev, double outlier, int drop_k, double* est_out);

/* One fixed-point step per (cell, technique): q^RR, q^S per channel from the
 * statistics, V_I and C_I.  Keeps previous values where n < 2, cost = 0 or
 * V_I <= 1e-12.  q_* and valid are updated in place. */
void orc_update_counts(int n_cells, int techniques, const double* stats, double VI, double CI,
                       float* q_rr, float* q_s, uint8_t* valid);

/* Guide update: per cell, P_b = 0.9 h_b / H + 0.1 / 256 (uniform when H = 0),
 * cdf = inclusive prefix sum of P. */
void orc_guide_update(int n_cells, const double* hist, float* cdf);

/* Test hooks (the renderer does not call them): light subpath steps drawn by
 * the renderer's routines, and the light-side densities the whole-path weights
 * give them.  l: light index; y0: a point on it.
 * orc_debug_light_emit: n cosine emission directions from y0, drawn by
 *   u[2i], u[2i+1]; hit[3i..3i+2] = the first hit, prim[i] its primitive (-1:
 *   miss).
 * orc_debug_light_bounce: y_1 = the first hit of the ray from y0 along d1; n
 *   bounces at y_1 (BSDF sampling and the roulette) drawn by u[3i..3i+2];
 *   hit / prim of the next vertex (-1: the subpath ended or missed).
 * orc_debug_light_density: out[0] = P<- of y_1 (emission density, area measure),
 *   out[1] = P<- of the first hit x' of the ray from y_1 towards x (the bounce
 *   density with the light arriving from y0, times the survival probability).
 * Return 0, or a negative value on invalid input (-4: the ray along d1 misses). */
int orc_debug_light_emit(const orc_scene_desc* scene, const orc_params* P, int l, const double* y0, int n,
                         const double* u, double* hit, int32_t* prim);
int orc_debug_light_bounce(const orc_scene_desc* scene, const orc_params* P, int l, const double* y0,
                           const double* d1, int n, const double* u, double* hit, int32_t* prim);
int orc_debug_light_density(const orc_scene_desc* scene, const orc_params* P, int l, const double* y0,
                            const double* d1, const double* x, double* out);

/* Adaptive octree cache (the spatial structure of EARS, Sec. 5.1), refined
 * between iterations.  Depth at most ORC_OCT_LMAX; a point's leaf is found by
 * descending with the bits of its cell coordinates at the finest level,
 * floor((p - lo) / ext * 2^LMAX) per axis decided in float32, octant =
 * x | y << 1 | z << 2.
 * orc_octree_init: the full tree down to the uniform grid (grid_n = 2^L0),
 *   leaves numbered like the grid's cells, (z * N + y) * N + x; nodes in
 *   breadth-first order.  Returns the node count.
 * orc_octree_refine: leaves in id order whose samples this iteration (n summed
 *   over the techniques, from stats) reach split_samples and whose level is
 *   below ORC_OCT_LMAX split into 8 while the leaf count stays <= max_leaves.
 *   Split s (0-based, in that order) turns node leaf_node[L] into an internal
 *   node with children at n_nodes + 8 s .. + 7; octant 0 keeps cell L, octant
 *   o > 0 gets the new cell n_leaves + 7 s + o - 1, which inherits L's counts
 *   (q, valid) and guide histogram and CDF.  Updates the counts in place and
 *   returns the number of splits. */
#define ORC_OCT_LMAX 10
/* leaf of the octree holding point p (scene box lo, ext) */
int orc_octree_cell(const double lo[3], const double ext[3], const int32_t* nodes, const double p[3]);
int orc_octree_init(int grid_n, int32_t* nodes, int32_t* leaf_level, int32_t* leaf_node);
int orc_octree_refine(int max_leaves, double split_samples, const double* stats, int32_t* nodes,
                      int32_t* n_nodes, int32_t* n_leaves, int32_t* leaf_level, int32_t* leaf_node,
                      float* q_rr, float* q_s, uint8_t* valid, double* hist, float* cdf);

/* Philox4x32-10 block for counter ctr[4] and key key[2]. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Alg. 1 (low-discrepancy stochastic rounding) in float32. */
void orc_stochastic_round(int n, const float* beta, float r, int32_t* gamma);

/* Count rule of the spatial update for one vertex: beta from q^RR, q^S (per
 * channel), throughput T and pixel estimate I, followed by the clamp. */
double orc_vertex_count(const float* q_rr, const float* q_s, const double* T, const float* I,
                        double lo, double hi);

/* Multi-sample balance heuristic weight of technique t among n techniques
 * (budget-aware when aware != 0). */
double orc_balance_weight(int n, const double* beta, const double* pdf, const int* participates,
                          int t, int aware);

/* BSDF helpers for tests: evaluate f*cos and the sampling pdf of material m in
 * a local frame (normal = +z), and draw one sample from uniforms u0, u1. */
void orc_bsdf_eval_local(const orc_scene_desc* scene, int m, const double* wo, const double* wi,
                         double* fcos_rgb, double* pdf);
int orc_bsdf_sample_local(const orc_scene_desc* scene, int m, const double* wo, double u0,
                          double u1, double* wi, double* pdf);
/* Guide pdf / sample for one cell's CDF (world directions). */
double orc_guide_pdf(const float* cdf, const double* w);
void orc_guide_sample(const float* cdf, double u0, double u1, double u2, double* w, double* pdf);

#ifdef __cplusplus
}
#endif
#endif
