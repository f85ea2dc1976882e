/*
 * mars_oracle.c -- plain, slow, single-threaded CPU oracle for MARS
 * (Meyer, Rath, Yazici, Slusallek, SIGGRAPH Asia 2024).
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA path and is loaded by the
 * tests, the smoke check and the benchmark's CPU-baseline leg, nothing else.
 * It shares no code with the CUDA path.  Build: gcc -O2 -ffp-contract=off.
 *
 * The renderer is a depth-first recursion that evaluates the paper's
 * estimators literally:
 *   - multi-sample MIS estimator with real-valued budgets (Eq. 1, Sec. 3),
 *   - per-vertex secondary estimator of reflected radiance (Sec. 3.1,
 *     "Secondary estimator"), primary estimator per technique ("Primary
 *     estimator"), random walk from the camera ("Random walks"),
 *   - budget-aware balance heuristic (Sec. 3 "Proxy model"; App. A.1 gives the
 *     budget-unaware form),
 *   - low-discrepancy stochastic rounding (Alg. 1, App. B.1),
 *   - spatially varying count update with throughput T(x)/I_px (Sec. 3.1
 *     "Optimization"), local estimates per cache cell (Sec. 4.1 "Local
 *     estimates"), image variance and cost (Sec. 4.1 "Image estimates"),
 *     outlier and count clamping (Sec. 4.1 "Outlier clamping"), channel
 *     handling ("Handling colors").
 * Readings of passages the paper leaves open are stated where they are used.
 *
 * The Philox bits are pinned by the generator's published known-answer
 * vectors; the light-side densities of the whole-path weights by brute force
 * (the landing frequencies of light subpath steps drawn by this renderer's own
 * routines, through the test hooks at the end of the file).
 */
#include "mars_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------ vectors */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 nrm(v3 a) { return scl(a, 1.0 / len(a)); }
static v3 ld3(const double* p) { return mk(p[0], p[1], p[2]); }

/* ------------------------------------------------------------ Philox4x32-10
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC 2011): ten rounds of two 32x32->64 multiplications with round keys
 * k + r * (0x9E3779B9, 0xBB67AE85). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* RNG keying (a reading; the paper uses an unspecified sampler):
 * key = (seed, job); counter = (pixel, iteration << 16 | dimension,
 * lineage low word, lineage high word).  Dimension: technique slot * 32 +
 * sample index for technique samples, 96 for the Alg. 1 draw, 97 for the
 * camera jitter, 128 + 8 s + k for step k of the light subpath of light
 * connection sample s (k = 0: light and point, 1: emission direction, k >= 2:
 * the bounce at the subpath's (k - 1)-th surface vertex and its Russian
 * roulette).  Each uniform takes the top 24 bits of one output word. */
enum { DIM_ROUND = 96, DIM_CAMERA = 97, DIM_LIGHT = 128 };
static void rng4(const orc_params* P, uint32_t px, uint32_t dim, uint64_t lin, double u[4]) {
  uint32_t ctr[4] = {px, (P->iteration << 16) | dim, (uint32_t)lin, (uint32_t)(lin >> 32)};
  uint32_t key[2] = {P->seed, P->job};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  for (int i = 0; i < 4; ++i) u[i] = (double)(o[i] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------- scene */
typedef struct {
  const orc_scene_desc* d;
  double lo[3], ext[3];
  double eps;
  int n_lights;
  int* light_quad;     /* quad index of light l */
  double* light_pmf;   /* selection probability of light l */
  float* light_cdf;    /* inclusive CDF, rounded to float */
  double tanh, aspect;
  v3 cam_o, cam_f, cam_r, cam_u;
  int bits;            /* lineage bits per level */
} ctx_t;

static const double* mat_of(const orc_scene_desc* d, int m) { return d->materials + 8 * m; }
static double mean3(const double* c) { return (c[0] + c[1] + c[2]) / 3.0; }

static void bbox_add(double lo[3], double hi[3], v3 p) {
  double a[3] = {p.x, p.y, p.z};
  for (int i = 0; i < 3; ++i) {
    if (a[i] < lo[i]) lo[i] = a[i];
    if (a[i] > hi[i]) hi[i] = a[i];
  }
}

static int ctx_init(ctx_t* C, const orc_scene_desc* d, const orc_params* P) {
  memset(C, 0, sizeof(*C));
  C->d = d;
  if (d->width <= 0 || d->height <= 0) return -1;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < d->n_quads; ++i) {
    const double* q = d->quads + 9 * i;
    v3 p0 = ld3(q), e1 = ld3(q + 3), e2 = ld3(q + 6);
    bbox_add(lo, hi, p0); bbox_add(lo, hi, add(p0, e1));
    bbox_add(lo, hi, add(p0, e2)); bbox_add(lo, hi, add(add(p0, e1), e2));
  }
  for (int i = 0; i < d->n_spheres; ++i) {
    const double* s = d->spheres + 4 * i;
    bbox_add(lo, hi, mk(s[0] - s[3], s[1] - s[3], s[2] - s[3]));
    bbox_add(lo, hi, mk(s[0] + s[3], s[1] + s[3], s[2] + s[3]));
  }
  for (int i = 0; i < d->n_tris; ++i)
    for (int k = 0; k < 3; ++k) bbox_add(lo, hi, ld3(d->tris + 9 * i + 3 * k));
  if (d->n_quads + d->n_spheres + d->n_tris == 0) return -1;
  double emax = 0.0;
  for (int i = 0; i < 3; ++i) {
    C->lo[i] = lo[i];
    C->ext[i] = hi[i] - lo[i] > 0.0 ? hi[i] - lo[i] : 1.0;
    if (hi[i] - lo[i] > emax) emax = hi[i] - lo[i];
  }
  /* ray offset: 1e-4 x the largest scene extent along the shading normal */
  C->eps = 1e-4 * (emax > 0.0 ? emax : 1.0);

  /* emitters: only quads may emit; one-sided along normalize(e1 x e2) */
  for (int i = 0; i < d->n_spheres; ++i)
    if (mean3(mat_of(d, d->sphere_mat[i]) + 5) > 0.0) return -1;
  for (int i = 0; i < d->n_tris; ++i)
    if (mean3(mat_of(d, d->tri_mat[i]) + 5) > 0.0) return -1;
  C->light_quad = (int*)malloc(sizeof(int) * (d->n_quads + 1));
  C->light_pmf = (double*)malloc(sizeof(double) * (d->n_quads + 1));
  C->light_cdf = (float*)malloc(sizeof(float) * (d->n_quads + 1));
  double tot = 0.0;
  for (int i = 0; i < d->n_quads; ++i) {
    const double* m = mat_of(d, d->quad_mat[i]);
    double p = mean3(m + 5);
    if (p > 0.0) {
      const double* q = d->quads + 9 * i;
      double area = len(cross(ld3(q + 3), ld3(q + 6)));
      C->light_quad[C->n_lights] = i;
      C->light_pmf[C->n_lights] = area * p; /* selection proportional to area x radiance */
      tot += area * p;
      C->n_lights++;
    }
  }
  double run = 0.0;
  for (int l = 0; l < C->n_lights; ++l) {
    run += C->light_pmf[l];
    C->light_pmf[l] /= tot;
    C->light_cdf[l] = (float)(run / tot);
  }
  if ((P->techniques & 2) && C->n_lights == 0) return -1;

  /* pinhole camera: right = normalize(up x forward), true up = forward x right */
  v3 o = ld3(d->camera), at = ld3(d->camera + 3), up = ld3(d->camera + 6);
  C->cam_o = o;
  C->cam_f = nrm(sub(at, o));
  C->cam_r = nrm(cross(up, C->cam_f));
  C->cam_u = cross(C->cam_f, C->cam_r);
  C->tanh = tan(0.5 * d->camera[9] * PI / 180.0);
  C->aspect = (double)d->width / (double)d->height;
  C->bits = (P->techniques & 4) ? 6 : 5;
  return 0;
}

static void ctx_free(ctx_t* C) {
  free(C->light_quad);
  free(C->light_pmf);
  free(C->light_cdf);
}

/* -------------------------------------------------------------- intersection */
typedef struct {
  double t;
  int prim;    /* global index: quads, then spheres, then triangles */
  v3 p, ng;    /* position, unit geometric normal */
  int mat;
} hit_t;

static int isect_quad(const double* q, v3 o, v3 d, double tmax, double* t_out) {
  v3 p0 = ld3(q), e1 = ld3(q + 3), e2 = ld3(q + 6);
  v3 n = cross(e1, e2);
  double den = dot(d, n);
  if (den == 0.0) return 0;
  double t = dot(sub(p0, o), n) / den;
  if (!(t > 0.0 && t < tmax)) return 0;
  v3 w = sub(add(o, scl(d, t)), p0);
  double nn = dot(n, n);
  double a = dot(cross(w, e2), n) / nn;
  double b = dot(cross(e1, w), n) / nn;
  if (a < 0.0 || a > 1.0 || b < 0.0 || b > 1.0) return 0;
  *t_out = t;
  return 1;
}

static int isect_sphere(const double* s, v3 o, v3 d, double tmax, double* t_out) {
  v3 oc = sub(o, ld3(s));
  double b = dot(oc, d);
  double c = dot(oc, oc) - s[3] * s[3];
  double disc = b * b - c;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double t = -b - sq;
  if (!(t > 0.0)) t = -b + sq;
  if (!(t > 0.0 && t < tmax)) return 0;
  *t_out = t;
  return 1;
}

static int isect_tri(const double* v, v3 o, v3 d, double tmax, double* t_out) {
  v3 v0 = ld3(v), e1 = sub(ld3(v + 3), v0), e2 = sub(ld3(v + 6), v0);
  v3 p = cross(d, e2);
  double det = dot(e1, p);
  if (det == 0.0) return 0;
  double inv = 1.0 / det;
  v3 s = sub(o, v0);
  double a = dot(s, p) * inv;
  if (a < 0.0 || a > 1.0) return 0;
  v3 q = cross(s, e1);
  double b = dot(d, q) * inv;
  if (b < 0.0 || a + b > 1.0) return 0;
  double t = dot(e2, q) * inv;
  if (!(t > 0.0 && t < tmax)) return 0;
  *t_out = t;
  return 1;
}

/* brute force over all primitives; the lowest index wins a tie in t */
static int closest_hit(const ctx_t* C, v3 o, v3 d, hit_t* h) {
  const orc_scene_desc* S = C->d;
  double best = INFINITY, t;
  int bi = -1;
  for (int i = 0; i < S->n_quads; ++i)
    if (isect_quad(S->quads + 9 * i, o, d, best, &t)) { best = t; bi = i; }
  for (int i = 0; i < S->n_spheres; ++i)
    if (isect_sphere(S->spheres + 4 * i, o, d, best, &t)) { best = t; bi = S->n_quads + i; }
  for (int i = 0; i < S->n_tris; ++i)
    if (isect_tri(S->tris + 9 * i, o, d, best, &t)) { best = t; bi = S->n_quads + S->n_spheres + i; }
  if (bi < 0) return 0;
  h->t = best;
  h->prim = bi;
  h->p = add(o, scl(d, best));
  if (bi < S->n_quads) {
    const double* q = S->quads + 9 * bi;
    h->ng = nrm(cross(ld3(q + 3), ld3(q + 6)));
    h->mat = S->quad_mat[bi];
  } else if (bi < S->n_quads + S->n_spheres) {
    int k = bi - S->n_quads;
    const double* s = S->spheres + 4 * k;
    h->ng = scl(sub(h->p, ld3(s)), 1.0 / s[3]);
    h->mat = S->sphere_mat[k];
  } else {
    int k = bi - S->n_quads - S->n_spheres;
    const double* v = S->tris + 9 * k;
    h->ng = nrm(cross(sub(ld3(v + 3), ld3(v)), sub(ld3(v + 6), ld3(v))));
    h->mat = S->tri_mat[k];
  }
  return 1;
}

static int occluded(const ctx_t* C, v3 o, v3 d, double tmax) {
  const orc_scene_desc* S = C->d;
  double t;
  for (int i = 0; i < S->n_quads; ++i)
    if (isect_quad(S->quads + 9 * i, o, d, tmax, &t)) return 1;
  for (int i = 0; i < S->n_spheres; ++i)
    if (isect_sphere(S->spheres + 4 * i, o, d, tmax, &t)) return 1;
  for (int i = 0; i < S->n_tris; ++i)
    if (isect_tri(S->tris + 9 * i, o, d, tmax, &t)) return 1;
  return 0;
}

/* ------------------------------------------------------------------- frames */
/* orthonormal basis around n (Duff et al., "Building an Orthonormal Basis,
 * Revisited", JCGT 2017) */
static void onb(v3 n, v3* b1, v3* b2) {
  double sign = copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *b1 = mk(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *b2 = mk(b, sign + n.y * n.y * a, -n.y);
}
static v3 to_world(v3 l, v3 b1, v3 b2, v3 n) {
  return add(add(scl(b1, l.x), scl(b2, l.y)), scl(n, l.z));
}
static v3 to_local(v3 w, v3 b1, v3 b2, v3 n) { return mk(dot(w, b1), dot(w, b2), dot(w, n)); }

/* ---------------------------------------------------------------------- BSDF
 * Lambert: f = albedo / pi, cosine-weighted sampling.
 * GGX (Walter et al. 2007): D(h) with roughness alpha, height-correlated Smith
 * masking-shadowing, Schlick Fresnel with F0 = material colour; sampling of
 * D(h) cos(theta_h) and reflection about h. */
static double ggx_D(double a2, double cz) {
  double k = cz * cz * (a2 - 1.0) + 1.0;
  return a2 / (PI * k * k);
}
static double ggx_Lambda(double a2, double cz) {
  double c2 = cz * cz;
  double t2 = (1.0 - c2) / c2;
  return 0.5 * (-1.0 + sqrt(1.0 + a2 * t2));
}

/* f(wo, wi) |cos theta_i| and the BSDF-sampling pdf of wi (local frame, n=+z) */
static void bsdf_eval(const double* m, v3 wo, v3 wi, double fcos[3], double* pdf) {
  fcos[0] = fcos[1] = fcos[2] = 0.0;
  *pdf = 0.0;
  if (wo.z <= 0.0 || wi.z <= 0.0) return;
  if ((int)m[0] == 0) {
    for (int c = 0; c < 3; ++c) fcos[c] = m[1 + c] / PI * wi.z;
    *pdf = wi.z / PI;
    return;
  }
  double a2 = m[4] * m[4];
  v3 h = nrm(add(wo, wi));
  double woh = dot(wo, h);
  if (woh <= 0.0) return;
  double D = ggx_D(a2, h.z);
  double G = 1.0 / (1.0 + ggx_Lambda(a2, wo.z) + ggx_Lambda(a2, wi.z));
  double s = 1.0 - woh;
  double s5 = s * s * s * s * s;
  for (int c = 0; c < 3; ++c) {
    double F = m[1 + c] + (1.0 - m[1 + c]) * s5;
    fcos[c] = D * G * F / (4.0 * wo.z);
  }
  *pdf = D * h.z / (4.0 * woh);
}

/* returns 1 and a direction with wi.z > 0 on success, 0 for an invalid sample */
static int bsdf_sample(const double* m, v3 wo, double u0, double u1, v3* wi) {
  if ((int)m[0] == 0) {
    double r = sqrt(u0), phi = 2.0 * PI * u1;
    double z = 1.0 - u0;
    *wi = mk(r * cos(phi), r * sin(phi), sqrt(z > 0.0 ? z : 0.0));
    return wi->z > 0.0;
  }
  double a2 = m[4] * m[4];
  double t2 = a2 * u0 / (1.0 - u0);
  double ct = 1.0 / sqrt(1.0 + t2);
  double st = sqrt(t2) * ct;
  double phi = 2.0 * PI * u1;
  v3 h = mk(st * cos(phi), st * sin(phi), ct);
  double woh = dot(wo, h);
  if (woh <= 0.0) return 0;
  *wi = sub(scl(h, 2.0 * woh), wo);
  return wi->z > 0.0;
}

void orc_bsdf_eval_local(const orc_scene_desc* scene, int m, const double* wo, const double* wi,
                         double* fcos_rgb, double* pdf) {
  bsdf_eval(mat_of(scene, m), ld3(wo), ld3(wi), fcos_rgb, pdf);
}

int orc_bsdf_sample_local(const orc_scene_desc* scene, int m, const double* wo, double u0,
                          double u1, double* wi, double* pdf) {
  v3 w;
  const double* mm = mat_of(scene, m);
  if (!bsdf_sample(mm, ld3(wo), u0, u1, &w)) { *pdf = 0.0; return 0; }
  double f[3];
  bsdf_eval(mm, ld3(wo), w, f, pdf);
  wi[0] = w.x; wi[1] = w.y; wi[2] = w.z;
  return 1;
}

/* ------------------------------------------------------------------- guide
 * Per-cell directional histogram on the cylinder (z = cos theta, phi), 16 x 16
 * equal-area bins; the bin index of a direction is decided in float32. */
static int guide_bin(v3 w) {
  float zf = (float)w.z;
  int iz = (int)floorf((zf + 1.0f) * 8.0f);
  if (iz < 0) iz = 0;
  if (iz > 15) iz = 15;
  float ph = atan2f((float)w.y, (float)w.x);
  if (ph < 0.0f) ph += 6.28318530717958647692f;
  int ip = (int)floorf(ph * (float)(16.0 / (2.0 * PI)));
  if (ip < 0) ip = 0;
  if (ip > 15) ip = 15;
  return iz * 16 + ip;
}
static double bin_prob(const float* cdf, int b) {
  float pb = cdf[b] - (b > 0 ? cdf[b - 1] : 0.0f); /* float subtraction on purpose */
  return (double)pb;
}
double orc_guide_pdf(const float* cdf, const double* w) {
  return bin_prob(cdf, guide_bin(ld3(w))) * (ORC_GUIDE_BINS / (4.0 * PI));
}
static int guide_pick(const float* cdf, float u0) {
  for (int b = 0; b < ORC_GUIDE_BINS; ++b)
    if (u0 < cdf[b]) return b;
  return ORC_GUIDE_BINS - 1;
}
static v3 guide_dir(int b, double u1, double u2) {
  int iz = b / 16, ip = b % 16;
  double z = -1.0 + 2.0 * ((double)iz + u1) / 16.0;
  double phi = 2.0 * PI * ((double)ip + u2) / 16.0;
  double s = 1.0 - z * z;
  s = sqrt(s > 0.0 ? s : 0.0);
  return mk(s * cos(phi), s * sin(phi), z);
}
void orc_guide_sample(const float* cdf, double u0, double u1, double u2, double* w, double* pdf) {
  int b = guide_pick(cdf, (float)u0);
  v3 d = guide_dir(b, u1, u2);
  w[0] = d.x; w[1] = d.y; w[2] = d.z;
  *pdf = bin_prob(cdf, b) * (ORC_GUIDE_BINS / (4.0 * PI));
}

/* --------------------------------------------------------- MIS and rounding */
/* Balance heuristic over the techniques that participate in a subintegrand
 * (App. A.1); budget-aware weights multiply each density by its real-valued
 * budget beta (reading of Sec. 3 "Proxy model": weights "containing the
 * techniques' budgets"). */
double orc_balance_weight(int n, const double* beta, const double* pdf, const int* participates,
                          int t, int aware) {
  double den = 0.0;
  for (int k = 0; k < n; ++k)
    if (participates[k]) den += (aware ? beta[k] : 1.0) * pdf[k];
  if (!participates[t] || den <= 0.0) return 0.0;
  return (aware ? beta[t] : 1.0) * pdf[t] / den;
}

/* Alg. 1: one uniform r decides the rounding of all techniques in order. */
void orc_stochastic_round(int n, const float* beta, float r, int32_t* gamma) {
  for (int t = 0; t < n; ++t) {
    float s = beta[t] + r;
    int32_t g = (int32_t)floorf(s);
    gamma[t] = g;
    r = s - (float)g;
  }
}

/* Spatial count (Sec. 3.1 "Optimization"; colour per "Handling colors"):
 * per channel beta_ch = T_ch / I_ch * q_ch for the RR and S factors, combined
 * by the root mean square over channels, then the three cases of the update
 * (RR if below 1, else S if above 1, else 1), then the clamp (Sec. 4.1). */
double orc_vertex_count(const float* q_rr, const float* q_s, const double* T, const float* I,
                        double lo, double hi) {
  double brr = 0.0, bs = 0.0;
  for (int c = 0; c < 3; ++c) {
    double f = T[c] / (double)I[c];
    double a = f * (double)q_rr[c], b = f * (double)q_s[c];
    brr += a * a;
    bs += b * b;
  }
  brr = sqrt(brr / 3.0);
  bs = sqrt(bs / 3.0);
  double beta = brr < 1.0 ? brr : (bs > 1.0 ? bs : 1.0);
  if (beta < lo) beta = lo;
  if (beta > hi) beta = hi;
  return beta;
}

/* ----------------------------------------------------------------- renderer */
/* A vertex of a full path in camera order (bidirectional application): its
 * position, unit geometric normal and material, the unit directions towards
 * the previous vertex (dp, towards the camera) and the next one (dn, towards
 * the light), and the distance tn to the next vertex. */
typedef struct {
  v3 p, ng, dp, dn;
  int mat;
  double tn;
} pathv_t;
#define ORC_MAXP 32

typedef struct {
  const ctx_t* C;
  const orc_params* P;
  orc_state* st;
  int px;
  int on[ORC_NT];  /* technique enabled */
  int bd;          /* bidirectional application: slot 2 is the light connection */
  /* the camera vertices x_1..x_k of the path being traced, index = depth; dn and
   * tn of x_j are those of the segment towards x_{j+1} (set before it is traced) */
  pathv_t cam[ORC_MAXP];
} rnd_t;

static void cell_coords(const ctx_t* C, int N, v3 p, int idx[3]) {
  /* the cell coordinates are decided in float32 */
  float pf[3] = {(float)p.x, (float)p.y, (float)p.z};
  for (int a = 0; a < 3; ++a) {
    float f = (pf[a] - (float)C->lo[a]) / (float)C->ext[a] * (float)N;
    int i = (int)floorf(f);
    if (i < 0) i = 0;
    if (i > N - 1) i = N - 1;
    idx[a] = i;
  }
}

static int cell_of(const ctx_t* C, int N, v3 p) {
  int idx[3];
  cell_coords(C, N, p, idx);
  return (idx[2] * N + idx[1]) * N + idx[0];
}

/* leaf of the adaptive octree holding p: descend with the bits of the point's
 * coordinates at the finest level, most significant first */
static int octree_cell(const ctx_t* C, const int32_t* nodes, v3 p) {
  int idx[3];
  cell_coords(C, 1 << ORC_OCT_LMAX, p, idx);
  int k = 0;
  for (int level = 0; level < ORC_OCT_LMAX && nodes[k] >= 0; ++level) {
    int sh = ORC_OCT_LMAX - 1 - level;
    int oct = ((idx[0] >> sh) & 1) | (((idx[1] >> sh) & 1) << 1) | (((idx[2] >> sh) & 1) << 2);
    k = nodes[k] + oct;
  }
  return ~nodes[k];
}

int orc_octree_cell(const double lo[3], const double ext[3], const int32_t* nodes, const double p[3]) {
  ctx_t C;
  memset(&C, 0, sizeof(C));
  for (int a = 0; a < 3; ++a) {
    C.lo[a] = lo[a];
    C.ext[a] = ext[a];
  }
  v3 q = {p[0], p[1], p[2]};
  return octree_cell(&C, nodes, q);
}

int orc_octree_init(int grid_n, int32_t* nodes, int32_t* leaf_level, int32_t* leaf_node) {
  int L0 = 0;
  while ((1 << L0) < grid_n) ++L0;
  if ((1 << L0) != grid_n || L0 > ORC_OCT_LMAX) return -1;
  /* breadth first: level l holds 8^l nodes; node (l, x, y, z) */
  int first = 0, count = 1, next = 1;
  int* cx = (int*)malloc(sizeof(int) * 3 * (size_t)grid_n * grid_n * grid_n + 3);
  cx[0] = cx[1] = cx[2] = 0;
  int* nx = (int*)malloc(sizeof(int) * 3 * (size_t)grid_n * grid_n * grid_n + 3);
  for (int l = 0; l <= L0; ++l) {
    for (int k = 0; k < count; ++k) {
      int x = cx[3 * k], y = cx[3 * k + 1], z = cx[3 * k + 2];
      if (l == L0) {
        int cell = (z * grid_n + y) * grid_n + x;
        nodes[first + k] = ~cell;
        leaf_level[cell] = L0;
        leaf_node[cell] = first + k;
      } else {
        nodes[first + k] = next + 8 * k;
        for (int o = 0; o < 8; ++o) {
          nx[3 * (8 * k + o)] = 2 * x + (o & 1);
          nx[3 * (8 * k + o) + 1] = 2 * y + ((o >> 1) & 1);
          nx[3 * (8 * k + o) + 2] = 2 * z + ((o >> 2) & 1);
        }
      }
    }
    if (l < L0) {
      first = next;
      next += 8 * count;
      count *= 8;
      int* t = cx;
      cx = nx;
      nx = t;
    }
  }
  free(cx);
  free(nx);
  return next;
}

int orc_octree_refine(int max_leaves, double split_samples, const double* stats, int32_t* nodes,
                      int32_t* n_nodes, int32_t* n_leaves, int32_t* leaf_level, int32_t* leaf_node,
                      float* q_rr, float* q_s, uint8_t* valid, double* hist, float* cdf) {
  const int L_count = *n_leaves, N0 = *n_nodes;
  const int budget = (max_leaves - L_count) / 7;
  int s = 0;
  for (int L = 0; L < L_count && s < budget; ++L) {
    double n = 0.0;
    for (int t = 0; t < ORC_NT; ++t) n += stats[((size_t)L * ORC_NT + t) * ORC_NSTAT];
    if (!(n >= split_samples) || leaf_level[L] >= ORC_OCT_LMAX) continue;
    const int base = N0 + 8 * s;
    nodes[leaf_node[L]] = base;
    nodes[base] = ~L;
    leaf_node[L] = base;
    leaf_level[L] += 1;
    for (int o = 1; o < 8; ++o) {
      const int c = L_count + 7 * s + o - 1;
      nodes[base + o] = ~c;
      leaf_node[c] = base + o;
      leaf_level[c] = leaf_level[L];
      for (int k = 0; k < ORC_NT * 3; ++k) {
        q_rr[(size_t)c * ORC_NT * 3 + k] = q_rr[(size_t)L * ORC_NT * 3 + k];
        q_s[(size_t)c * ORC_NT * 3 + k] = q_s[(size_t)L * ORC_NT * 3 + k];
      }
      for (int t = 0; t < ORC_NT; ++t) valid[(size_t)c * ORC_NT + t] = valid[(size_t)L * ORC_NT + t];
      if (hist && cdf)
        for (int b = 0; b < ORC_GUIDE_BINS; ++b) {
          hist[(size_t)c * ORC_GUIDE_BINS + b] = hist[(size_t)L * ORC_GUIDE_BINS + b];
          cdf[(size_t)c * ORC_GUIDE_BINS + b] = cdf[(size_t)L * ORC_GUIDE_BINS + b];
        }
    }
    ++s;
  }
  *n_nodes = N0 + 8 * s;
  *n_leaves = L_count + 7 * s;
  return s;
}

static double lum(const double* c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

typedef struct {
  v3 p, ng, ns, wo;
  int mat, cell;
  v3 b1, b2;
} vtx_t;

static void secondary_estimator(rnd_t* R, const vtx_t* x, int depth, uint64_t lin, const double T[3],
                                float mult, double Lr[3], double* cost);

/* pdf of the NEE technique for a direction that reaches point y on light quad q */
static double nee_pdf_at(const ctx_t* C, int quad, v3 x, v3 y, v3 wi) {
  for (int l = 0; l < C->n_lights; ++l) {
    if (C->light_quad[l] != quad) continue;
    const double* q = C->d->quads + 9 * quad;
    v3 n = cross(ld3(q + 3), ld3(q + 6));
    double area = len(n);
    n = scl(n, 1.0 / area);
    double cosl = -dot(n, wi);
    if (cosl <= 0.0) return 0.0;
    v3 dv = sub(y, x);
    return C->light_pmf[l] * dot(dv, dv) / (area * cosl);
  }
  return 0.0;
}

/* ------------------------------------------- bidirectional application
 * Sec. 5 combines three techniques at every camera vertex, each with its own
 * budget: path tracing (the BSDF continuation), NEE, and connections to the
 * vertices of light subpaths ("light connection", slot 2).  Readings (the
 * paper gives no formulas for them):
 *  - one light connection sample at x_i traces one light subpath of its own:
 *    a light chosen as for NEE (area x radiance) with a uniform point y_0,
 *    a cosine-distributed emission direction, BSDF sampling at every surface
 *    vertex, throughput-based Russian roulette after each bounce (continue
 *    with probability q = min(1, max_ch f cos / p) and divide by it; Sec. 5:
 *    light paths are never split), at most ORC_LIGHT_MAX surface vertices and
 *    at most D - 1 - i (the full path keeps at most D segments); the sample
 *    connects x_i to every surface vertex y_1..y_m of it (y_0 is NEE's), and
 *    its value is the sum of the weighted connections;
 *  - a light connection sample is drawn only at vertices with i <= D - 2 (a
 *    connection from x_{D-1} would exceed D segments); its base budget is 1,
 *    as NEE's;
 *  - the weights are the balance heuristic over every strategy that samples
 *    the same full path z_1..z_n (z_n on a light): the camera path alone
 *    (BSDF sampling to z_n), NEE at z_{n-1}, and light connection at z_i for
 *    i = 1..n-2 with n - 1 - i <= ORC_LIGHT_MAX light surface vertices; each
 *    strategy's density is multiplied by its expected sample count, the
 *    product of the budgets of the camera vertices it passes through (BSDF
 *    budgets, then the budget of its last technique) -- budget-aware
 *    multi-sample MIS over whole paths (budget-unaware: every count 1); the
 *    budgets at vertices that a strategy would have reached as camera vertices
 *    are evaluated by the count rule there, with the throughput T of a camera
 *    path through them;
 *  - the BSDF continuation carries no MIS weight (w_ind = 1): every
 *    contribution is weighted once, where its full path ends;
 *  - the local outlier clamp is off (Sec. 5.1: local outlier rejection
 *    lowered efficiency in this application). */

/* light index of quad primitive q, -1 if it does not emit */
static int light_of_quad(const ctx_t* C, int q) {
  for (int l = 0; l < C->n_lights; ++l)
    if (C->light_quad[l] == q) return l;
  return -1;
}

/* end point of a full path: a point on light l */
typedef struct {
  int l;
  v3 p, n;     /* point, unit emitting normal */
  double pN;   /* area density of NEE's light point (pmf / area) */
} light_end;

static light_end light_end_at(const ctx_t* C, int l, v3 y) {
  light_end e;
  const double* q = C->d->quads + 9 * C->light_quad[l];
  v3 n = cross(ld3(q + 3), ld3(q + 6));
  double area = len(n);
  e.l = l;
  e.p = y;
  e.n = scl(n, 1.0 / area);
  e.pN = C->light_pmf[l] / area;
  return e;
}

/* f |cos wi| and the BSDF-sampling density of wi given wo at a path vertex,
 * the shading normal facing wo */
static void bsdf_at(const ctx_t* C, const pathv_t* z, v3 wo, v3 wi, double fc[3], double* pdf) {
  v3 ns = dot(z->ng, wo) >= 0.0 ? z->ng : scl(z->ng, -1.0);
  v3 b1, b2;
  onb(ns, &b1, &b2);
  bsdf_eval(mat_of(C->d, z->mat), to_local(wo, b1, b2, ns), to_local(wi, b1, b2, ns), fc, pdf);
}

static double max3(const double* a) { return fmax(a[0], fmax(a[1], a[2])); }

/* technique t drawn at a camera vertex of this depth */
static int tech_at(const rnd_t* R, int t, int depth) {
  if (!R->on[t]) return 0;
  if (R->bd && t == ORC_T_LIGHT && depth > R->P->max_depth - 2) return 0;
  return 1;
}

static int cell_at(const rnd_t* R, v3 p) {
  return R->st->oct_nodes ? octree_cell(R->C, R->st->oct_nodes, p) : cell_of(R->C, R->P->grid_n, p);
}

/* Budgets beta_t at a vertex of depth `depth` in `cell` with throughput T and
 * path multiplicity mult.  Without learned counts (warm-up, fixed-count mode,
 * cells without statistics) every vertex draws one NEE sample (and one light
 * connection sample) and one continuation sample split evenly over the
 * continuation techniques (BSDF, guided): Sec. 4.1 "Fixed-point iteration"
 * warms up without splitting; with two continuation techniques beta = 1 each
 * would double every path at every bounce.  Alg. 1 turns (1/2, 1/2) into
 * exactly one continuation.  With a multiplicity cap M > 0 every budget is
 * further limited to max(clamp_lo, M / mult) (in float32).  The budgets are
 * carried in float32. */
static void budgets_at(const rnd_t* R, int cell, int depth, const double T[3], float mult, float betaf[ORC_NT]) {
  const orc_params* P = R->P;
  const orc_state* st = R->st;
  const int guided = R->on[ORC_T_GUIDED] && !R->bd;
  const double base_cont = 1.0 / (double)(R->on[ORC_T_BSDF] + guided);
  for (int t = 0; t < ORC_NT; ++t) {
    betaf[t] = 0.0f;
    if (!tech_at(R, t, depth)) continue;
    double b = (t == ORC_T_NEE || (R->bd && t == ORC_T_LIGHT)) ? 1.0 : base_cont;
    if (P->mode == ORC_MODE_MARS && st->valid[cell * ORC_NT + t]) {
      size_t o = ((size_t)cell * ORC_NT + t) * 3;
      b = orc_vertex_count(st->q_rr + o, st->q_s + o, T, st->est + 3 * R->px, P->clamp_lo, P->clamp_hi);
    }
    betaf[t] = (float)b;
    if (P->max_mult > 0.0f) {
      float cap = P->max_mult / mult;
      if (cap < (float)P->clamp_lo) cap = (float)P->clamp_lo;
      if (betaf[t] > cap) betaf[t] = cap;
    }
  }
}

enum { STRAT_CAMERA = 0, STRAT_NEE = 1, STRAT_LIGHT = 2 };

/* P<-_j: the area density of path vertex z_j on a light subpath.  With z_{j+1}
 * (zj1): BSDF sampling at z_{j+1} with the light arriving from z_{j+2} (its dn)
 * towards z_j (its dp), times that bounce's survival probability q =
 * min(1, max_ch f cos / p); without (zj1 = NULL): cosine emission from the light
 * point of e.  The solid-angle density becomes an area density by |cos| at z_j
 * over the squared distance. */
static double light_side_density(const ctx_t* C, const pathv_t* zj, const pathv_t* zj1, const light_end* e) {
  double cos_j = fabs(dot(zj->ng, zj->dn)), g = cos_j / (zj->tn * zj->tn);
  if (!zj1) {
    double cl = -dot(e->n, zj->dn);
    return cl > 0.0 ? cl / PI * g : 0.0;
  }
  double fc[3], pB;
  bsdf_at(C, zj1, zj1->dn, zj1->dp, fc, &pB);
  double q = pB > 0.0 ? fmin(1.0, max3(fc) / pB) : 0.0;
  return pB * q * g;
}

/* Balance-heuristic weight, over every strategy that samples it, of the full
 * path z[1..n-1], e (camera order; z[0] unused), for the strategy `kind`
 * (STRAT_LIGHT: connection at camera vertex z[si]).  Evaluated from the
 * definitions, strategy by strategy:
 *   C_1 = 1, C_{j+1} = C_j bw_B(z_j) P->_j     (camera prefix: BSDF counts x densities)
 *   camera path: C_n;  NEE at z_{n-1}: C_{n-1} bw_N(z_{n-1}) pN;
 *   light connection at z_i: C_i bw_L(z_i) pN prod_{j=i+1}^{n-1} P<-_j,
 * with P->_j the area density of z_{j+1} by BSDF sampling at z_j, P<-_j the
 * area density of z_j on a light subpath (cosine emission from z_n, or BSDF
 * sampling at z_{j+1} towards z_j times its survival probability), pN the
 * area density of the light point, and bw = beta (budget-aware) or 1. */
static double path_weight(const rnd_t* R, int n, const pathv_t* z, const light_end* e, int kind, int si) {
  const ctx_t* C = R->C;
  const orc_params* P = R->P;
  const int aware = P->weights == ORC_WEIGHTS_AWARE;
  double CP[ORC_MAXP], LP[ORC_MAXP], bwN[ORC_MAXP], bwL[ORC_MAXP];
  double T[3] = {1.0, 1.0, 1.0};
  float mult = 1.0f;
  for (int j = 1; j <= n - 1; ++j) {
    float bf[ORC_NT];
    budgets_at(R, cell_at(R, z[j].p), j, T, mult, bf);
    double fc[3], pB;
    bsdf_at(C, &z[j], z[j].dp, z[j].dn, fc, &pB);
    double cos_next = j + 1 < n ? fabs(dot(z[j + 1].ng, z[j].dn)) : -dot(e->n, z[j].dn);
    if (cos_next < 0.0) cos_next = 0.0;
    CP[j] = (aware ? (double)bf[ORC_T_BSDF] : 1.0) * pB * cos_next / (z[j].tn * z[j].tn);
    bwN[j] = tech_at(R, ORC_T_NEE, j) ? (aware ? (double)bf[ORC_T_NEE] : 1.0) : 0.0;
    bwL[j] = tech_at(R, ORC_T_LIGHT, j) ? (aware ? (double)bf[ORC_T_LIGHT] : 1.0) : 0.0;
    for (int ch = 0; ch < 3; ++ch) T[ch] = pB > 0.0 ? T[ch] * fc[ch] / pB / (double)bf[ORC_T_BSDF] : 0.0;
    mult = mult * bf[ORC_T_BSDF];
  }
  for (int j = 1; j <= n - 1; ++j) LP[j] = light_side_density(C, &z[j], j == n - 1 ? NULL : &z[j + 1], e);
  double sum = 0.0, chosen = 0.0, Cj = 1.0;
  for (int j = 1; j <= n - 1; ++j) {
    /* light connection at z_j to z_{j+1} (n - 1 - j light surface vertices) */
    int k = n - 1 - j;
    if (R->bd && k >= 1 && k <= ORC_LIGHT_MAX && bwL[j] > 0.0) {
      double t = Cj * bwL[j] * e->pN;
      for (int m = j + 1; m <= n - 1; ++m) t *= LP[m];
      sum += t;
      if (kind == STRAT_LIGHT && si == j) chosen = t;
    }
    if (j == n - 1 && bwN[j] > 0.0) {
      double t = Cj * bwN[j] * e->pN;
      sum += t;
      if (kind == STRAT_NEE) chosen = t;
    }
    Cj *= CP[j];
  }
  sum += Cj;
  if (kind == STRAT_CAMERA) chosen = Cj;
  return sum > 0.0 ? chosen / sum : 0.0;
}

/* cosine-distributed direction about the unit normal n, drawn by (u0, u1) */
static v3 emit_dir(v3 n, double u0, double u1) {
  v3 b1, b2;
  onb(n, &b1, &b2);
  double r = sqrt(u0), phi = 2.0 * PI * u1, zc = 1.0 - u0;
  return to_world(mk(r * cos(phi), r * sin(phi), sqrt(zc > 0.0 ? zc : 0.0)), b1, b2, n);
}

/* One bounce of a light subpath at the hit h, the light arriving along l_in
 * (the unit direction towards the previous light vertex): BSDF sampling with
 * u[0], u[1], then throughput-based Russian roulette with u[2] (survival
 * q = min(1, max_ch f cos / p), decided in float32).  Returns 0 if the subpath
 * ends there; else the offset origin and direction of the next ray and the
 * throughput factor f cos / (p q). */
static int light_bounce(const ctx_t* C, const hit_t* h, v3 l_in, const double u[4], v3* org, v3* dir,
                        double wb[3]) {
  const double* mat = mat_of(C->d, h->mat);
  v3 ns = dot(h->ng, l_in) >= 0.0 ? h->ng : scl(h->ng, -1.0);
  v3 c1, c2;
  onb(ns, &c1, &c2);
  v3 wl;
  if (!bsdf_sample(mat, to_local(l_in, c1, c2, ns), u[0], u[1], &wl)) return 0;
  v3 o = to_world(wl, c1, c2, ns);
  double fc[3], pB;
  bsdf_eval(mat, to_local(l_in, c1, c2, ns), wl, fc, &pB);
  if (!(pB > 0.0) || !(fc[0] > 0.0 || fc[1] > 0.0 || fc[2] > 0.0)) return 0;
  double qk = fmin(1.0, max3(fc) / pB);
  if (!((float)u[2] < (float)qk)) return 0;
  for (int c = 0; c < 3; ++c) wb[c] = fc[c] / pB / qk;
  *org = add(h->p, scl(ns, C->eps));
  *dir = o;
  return 1;
}

/* one light connection sample at camera vertex x (depth i): its light subpath
 * and the weighted connections to it; returns the sample value and its cost
 * (the rays its subpath traced plus one per connection) */
static void light_connection(rnd_t* R, const vtx_t* x, int depth_i, uint64_t lin, int s, double v[3],
                             double* cost) {
  const ctx_t* C = R->C;
  const orc_params* P = R->P;
  orc_state* st = R->st;
  v[0] = v[1] = v[2] = 0.0;
  *cost = 0.0;
  int kmax = P->max_depth - 1 - depth_i;
  if (kmax > ORC_LIGHT_MAX) kmax = ORC_LIGHT_MAX;
  if (kmax < 1 || C->n_lights == 0) return;
  double u[4];
  /* y_0: light by area x radiance (decided in float32), uniform point */
  rng4(P, (uint32_t)R->px, (uint32_t)(DIM_LIGHT + 8 * s), lin, u);
  int l = C->n_lights - 1;
  for (int k = 0; k < C->n_lights; ++k)
    if ((float)u[0] < C->light_cdf[k]) { l = k; break; }
  const double* q = C->d->quads + 9 * C->light_quad[l];
  v3 y0 = add(ld3(q), add(scl(ld3(q + 3), u[1]), scl(ld3(q + 6), u[2])));
  light_end e = light_end_at(C, l, y0);
  const double* Le = mat_of(C->d, C->d->quad_mat[C->light_quad[l]]) + 5;
  /* cosine-distributed emission direction about the light's normal */
  rng4(P, (uint32_t)R->px, (uint32_t)(DIM_LIGHT + 8 * s + 1), lin, u);
  v3 dir = emit_dir(e.n, u[0], u[1]);
  v3 org = add(y0, scl(e.n, C->eps));
  /* alpha_1 = Le cos / (pN p_omega) = Le pi / pN */
  double alpha[3];
  for (int c = 0; c < 3; ++c) alpha[c] = Le[c] * PI / e.pN;
  pathv_t y[ORC_LIGHT_MAX + 1];
  double ya[ORC_LIGHT_MAX + 1][3];
  int m = 0, rays = 0;
  for (int k = 1; k <= kmax; ++k) {
    hit_t h;
    rays += 1;
    st->counters[1] += 1.0;
    st->counters[6] += 1.0;
    if (!closest_hit(C, org, dir, &h)) break;
    const double* mat = mat_of(C->d, h.mat);
    if (!(mat[1] > 0.0 || mat[2] > 0.0 || mat[3] > 0.0)) break;
    pathv_t* yk = &y[k];
    yk->p = h.p;
    yk->ng = h.ng;
    yk->mat = h.mat;
    yk->dn = scl(dir, -1.0);   /* camera order: towards y_{k-1} */
    yk->tn = h.t;
    for (int c = 0; c < 3; ++c) ya[k][c] = alpha[c];
    yk->dp = mk(0, 0, 0);      /* towards the camera side: set by the connection */
    m = k;
    if (k == kmax) break;
    /* continue: BSDF sampling at y_k with the light arriving from y_{k-1} */
    rng4(P, (uint32_t)R->px, (uint32_t)(DIM_LIGHT + 8 * s + k + 1), lin, u);
    double wb[3];
    if (!light_bounce(C, &h, yk->dn, u, &org, &dir, wb)) break;
    for (int c = 0; c < 3; ++c) alpha[c] *= wb[c];
  }
  *cost = (double)(rays + m);
  /* connections x_i -- y_k */
  v3 xo = add(x->p, scl(x->ns, C->eps));
  for (int k = 1; k <= m; ++k) {
    v3 nsy = dot(y[k].ng, y[k].dn) >= 0.0 ? y[k].ng : scl(y[k].ng, -1.0);
    v3 yo = add(y[k].p, scl(nsy, C->eps));
    v3 dv = sub(yo, xo);
    double dist = len(dv);
    v3 w = scl(dv, 1.0 / dist);
    double fx[3], px_, fy[3], py;
    bsdf_eval(mat_of(C->d, x->mat), to_local(x->wo, x->b1, x->b2, x->ns), to_local(w, x->b1, x->b2, x->ns), fx,
              &px_);
    pathv_t yv = y[k];
    yv.dp = scl(w, -1.0);
    bsdf_at(C, &yv, y[k].dn, scl(w, -1.0), fy, &py);
    double cval[3];
    int nz = 0;
    for (int c = 0; c < 3; ++c) {
      cval[c] = ya[k][c] * fy[c] * fx[c] / (dist * dist);
      nz |= cval[c] > 0.0;
    }
    if (!nz) continue;
    /* the full path: x_1..x_i, y_k..y_1, y_0 */
    pathv_t z[ORC_MAXP];
    for (int j = 1; j <= depth_i; ++j) z[j] = R->cam[j];
    z[depth_i].dn = w;
    z[depth_i].tn = dist;
    for (int a = 1; a <= k; ++a) {
      z[depth_i + a] = y[k - a + 1];
      z[depth_i + a].dp = a == 1 ? scl(w, -1.0) : scl(y[k - a + 2].dn, -1.0);
    }
    int n = depth_i + 1 + k;
    double wgt = path_weight(R, n, z, &e, STRAT_LIGHT, depth_i);
    st->counters[7] += 1.0;
    if (occluded(C, xo, w, dist - C->eps)) continue;
    for (int c = 0; c < 3; ++c) v[c] += wgt * cval[c];
  }
}

/* Trace a ray drawn at the parent (or the camera) and return its sample value
 * fcp * (Le * w_dir + w_ind * <L_r(child)>), its cost in rays, and the
 * luminance of the incident radiance estimate (for guide learning). */
typedef struct {
  double fcp[3];     /* f |cos| / p_t at the parent (1 for the camera) */
  double A;          /* MIS numerator of the drawing technique */
  double S_ind;      /* MIS denominator over the indirect techniques */
  double betaN_pN0;  /* beta_NEE (aware) or 1 (unaware) if NEE competes, else 0 */
  int camera;        /* camera ray: no MIS */
  double T_child[3]; /* prefix throughput at the hit */
  float mult_child;  /* path multiplicity at the hit (product of the budgets that drew the path) */
} ray_info;

static void trace_sample(rnd_t* R, v3 o, v3 d, int depth, uint64_t lin, const ray_info* ri,
                         double v_out[3], double* cost_out, double* Li_lum) {
  const ctx_t* C = R->C;
  const orc_params* P = R->P;
  hit_t h;
  double E[3] = {0, 0, 0}, Le_raw[3] = {0, 0, 0}, Lchild[3] = {0, 0, 0};
  double ccost = 0.0;
  double w_ind = ri->camera ? 1.0 : (ri->S_ind > 0.0 ? ri->A / ri->S_ind : 0.0);
  R->st->counters[1] += 1.0; /* one traced path vertex */
  if (closest_hit(C, o, d, &h)) {
    v3 wo = scl(d, -1.0);
    const double* m = mat_of(C->d, h.mat);
    double cosg = dot(h.ng, wo);
    if (!ri->camera && R->bd) {
      /* the parent's segment towards this hit */
      R->cam[depth - 1].dn = d;
      R->cam[depth - 1].tn = h.t;
    }
    if (cosg > 0.0 && mean3(m + 5) > 0.0) {
      /* emission reached by a technique sample: weight against NEE's density
       * (and, bidirectionally, against every strategy of the full path) */
      double w_dir = 1.0;
      if (!ri->camera && R->bd) {
        int l = h.prim < C->d->n_quads ? light_of_quad(C, h.prim) : -1;
        if (l >= 0) {
          light_end e = light_end_at(C, l, h.p);
          w_dir = path_weight(R, depth, R->cam, &e, STRAT_CAMERA, 0);
        }
      } else if (!ri->camera) {
        double pn = 0.0;
        if (ri->betaN_pN0 > 0.0 && h.prim < C->d->n_quads)
          pn = nee_pdf_at(C, h.prim, o, h.p, d);
        double den = ri->S_ind + ri->betaN_pN0 * pn;
        w_dir = den > 0.0 ? ri->A / den : 0.0;
      }
      for (int c = 0; c < 3; ++c) {
        Le_raw[c] = m[5 + c];
        E[c] = m[5 + c] * w_dir;
      }
    }
    int reflective = (m[1] > 0.0 || m[2] > 0.0 || m[3] > 0.0);
    if (depth <= P->max_depth - 1 && reflective) {
      vtx_t x;
      x.p = h.p;
      x.ng = h.ng;
      x.wo = wo;
      x.ns = cosg >= 0.0 ? h.ng : scl(h.ng, -1.0);
      x.mat = h.mat;
      x.cell = cell_at(R, h.p);
      onb(x.ns, &x.b1, &x.b2);
      secondary_estimator(R, &x, depth, lin, ri->T_child, ri->mult_child, Lchild, &ccost);
    }
  }
  for (int c = 0; c < 3; ++c) v_out[c] = ri->fcp[c] * (E[c] + w_ind * Lchild[c]);
  *cost_out = 1.0 + ccost;
  if (Li_lum) {
    double Li[3] = {Le_raw[0] + Lchild[0], Le_raw[1] + Lchild[1], Le_raw[2] + Lchild[2]};
    *Li_lum = lum(Li);
  }
}

static void stat_add(rnd_t* R, int cell, int t, const double v[3], double cost, const double T[3]) {
  if (!R->P->collect) return;
  double* s = R->st->stats + ((size_t)cell * ORC_NT + t) * ORC_NSTAT;
  s[0] += 1.0;
  for (int c = 0; c < 3; ++c) {
    double x = v[c];
    /* local outlier clamp (Sec. 4.1): the sample's image contribution is kept
     * below outlier x pixel estimate, i.e. v <= outlier * I_px / T (not in the
     * bidirectional application, Sec. 5.1) */
    if (R->P->has_estimate && T[c] > 0.0 && !R->bd) {
      double lim = R->P->outlier * (double)R->st->est[3 * R->px + c] / T[c];
      if (x > lim) x = lim;
    }
    s[1 + c] += x;
    s[4 + c] += x * x;
  }
  s[7] += cost;
}

/* Secondary estimator at vertex x (Sec. 3.1): sum over techniques t of
 * 1/beta_t times the sum of gamma_t primary estimates, gamma from Alg. 1.
 * mult is the path multiplicity at x: the product of the budgets of the
 * techniques that drew the path's earlier vertices (1 at the first vertex),
 * see budgets_at. */
static void secondary_estimator(rnd_t* R, const vtx_t* x, int depth, uint64_t lin, const double T[3],
                                float mult, double Lr[3], double* cost) {
  const ctx_t* C = R->C;
  const orc_params* P = R->P;
  orc_state* st = R->st;
  const double* m = mat_of(C->d, x->mat);
  Lr[0] = Lr[1] = Lr[2] = 0.0;
  *cost = 0.0;
  st->counters[2] += 1.0;
  if (R->bd) {
    R->cam[depth].p = x->p;
    R->cam[depth].ng = x->ng;
    R->cam[depth].dp = x->wo;
    R->cam[depth].mat = x->mat;
  }

  float betaf[ORC_NT];
  double beta[ORC_NT];
  budgets_at(R, x->cell, depth, T, mult, betaf);
  for (int t = 0; t < ORC_NT; ++t) {
    beta[t] = (double)betaf[t];
    st->counters[3 + t] += beta[t];
  }

  /* Alg. 1 over the techniques drawn at this vertex */
  double u[4];
  rng4(P, (uint32_t)R->px, DIM_ROUND, lin, u);
  float rb[ORC_NT];
  int32_t gam[ORC_NT];
  int n_on = 0, idx[ORC_NT];
  for (int t = 0; t < ORC_NT; ++t)
    if (tech_at(R, t, depth)) { rb[n_on] = betaf[t]; idx[n_on++] = t; }
  int32_t gtmp[ORC_NT];
  orc_stochastic_round(n_on, rb, (float)u[0], gtmp);
  for (int t = 0; t < ORC_NT; ++t) gam[t] = 0;
  for (int k = 0; k < n_on; ++k) gam[idx[k]] = gtmp[k];

  /* MIS participation: direct light {BSDF, NEE, guided}, indirect {BSDF, guided} */
  int aware = P->weights == ORC_WEIGHTS_AWARE;
  double bw[ORC_NT];
  for (int t = 0; t < ORC_NT; ++t) bw[t] = R->on[t] ? (aware ? beta[t] : 1.0) : 0.0;
  if (R->bd) bw[ORC_T_LIGHT] = 0.0;   /* not a direction-sampling technique */
  const float* cdf = (R->on[ORC_T_GUIDED] && !R->bd) ? st->guide_cdf + (size_t)x->cell * ORC_GUIDE_BINS : NULL;

  for (int t = 0; t < ORC_NT; ++t) {
    for (int s = 0; s < gam[t]; ++s) {
      double v[3] = {0, 0, 0}, c_s = 1.0;
      if (R->bd && t == ORC_T_LIGHT) {
        light_connection(R, x, depth, lin, s, v, &c_s);
        for (int c = 0; c < 3; ++c) Lr[c] += v[c] / beta[t];
        *cost += c_s;
        stat_add(R, x->cell, t, v, c_s, T);
        continue;
      }
      rng4(P, (uint32_t)R->px, (uint32_t)(t * 32 + s), lin, u);
      if (t == ORC_T_NEE) {
        /* primary estimator of NEE: light by area x radiance, uniform point */
        int l = C->n_lights - 1;
        for (int k = 0; k < C->n_lights; ++k)
          if ((float)u[0] < C->light_cdf[k]) { l = k; break; }
        int qi = C->light_quad[l];
        const double* q = C->d->quads + 9 * qi;
        v3 y = add(ld3(q), add(scl(ld3(q + 3), u[1]), scl(ld3(q + 6), u[2])));
        v3 xo = add(x->p, scl(x->ns, C->eps));
        v3 dv = sub(y, xo);
        double dist = len(dv);
        v3 wi = scl(dv, 1.0 / dist);
        double pn = nee_pdf_at(C, qi, xo, y, wi);
        double ci = dot(x->ns, wi);
        if (pn > 0.0 && ci > 0.0) {
          double fc[3], pb, pg = 0.0;
          bsdf_eval(m, to_local(x->wo, x->b1, x->b2, x->ns), to_local(wi, x->b1, x->b2, x->ns), fc, &pb);
          if (cdf) pg = orc_guide_pdf(cdf, (double[]){wi.x, wi.y, wi.z});
          if ((fc[0] > 0.0 || fc[1] > 0.0 || fc[2] > 0.0) && !occluded(C, xo, wi, dist - C->eps)) {
            double w;
            if (R->bd) {
              /* the full path x_1..x_depth, y: weight over every strategy */
              R->cam[depth].dn = wi;
              R->cam[depth].tn = dist;
              light_end e = light_end_at(C, l, y);
              w = path_weight(R, depth + 1, R->cam, &e, STRAT_NEE, 0);
            } else {
              double den = bw[ORC_T_BSDF] * pb + bw[ORC_T_GUIDED] * pg + bw[ORC_T_NEE] * pn;
              w = bw[ORC_T_NEE] * pn / den;
            }
            const double* Le = mat_of(C->d, C->d->quad_mat[qi]) + 5;
            for (int c = 0; c < 3; ++c) v[c] = fc[c] * Le[c] / pn * w;
          }
        }
      } else {
        /* primary estimator of BSDF or guided sampling: extend the path */
        v3 wi;
        int ok;
        double pt = 0.0;
        if (t == ORC_T_BSDF) {
          v3 wl;
          ok = bsdf_sample(m, to_local(x->wo, x->b1, x->b2, x->ns), u[0], u[1], &wl);
          if (ok) wi = to_world(wl, x->b1, x->b2, x->ns);
        } else {
          int b = guide_pick(cdf, (float)u[0]);
          wi = guide_dir(b, u[1], u[2]);
          pt = bin_prob(cdf, b) * (ORC_GUIDE_BINS / (4.0 * PI));
          ok = dot(wi, x->ns) > 0.0;
        }
        if (ok) {
          double fc[3], pb, pg = 0.0;
          bsdf_eval(m, to_local(x->wo, x->b1, x->b2, x->ns), to_local(wi, x->b1, x->b2, x->ns), fc, &pb);
          if (cdf) pg = orc_guide_pdf(cdf, (double[]){wi.x, wi.y, wi.z});
          if (t == ORC_T_BSDF) pt = pb;
          if (pt > 0.0 && (fc[0] > 0.0 || fc[1] > 0.0 || fc[2] > 0.0)) {
            ray_info ri;
            ri.camera = 0;
            for (int c = 0; c < 3; ++c) ri.fcp[c] = fc[c] / pt;
            ri.A = bw[t] * pt;
            ri.S_ind = bw[ORC_T_BSDF] * pb + bw[ORC_T_GUIDED] * pg;
            ri.betaN_pN0 = bw[ORC_T_NEE];
            double w_ind = ri.A / ri.S_ind;
            for (int c = 0; c < 3; ++c) ri.T_child[c] = T[c] * ri.fcp[c] * w_ind / beta[t];
            ri.mult_child = mult * betaf[t];
            uint64_t digit = (uint64_t)(t == ORC_T_BSDF ? s + 1 : 32 + s + 1);
            uint64_t clin = (lin << C->bits) | digit;
            double li_lum = 0.0;
            trace_sample(R, add(x->p, scl(x->ns, C->eps)), wi, depth + 1, clin, &ri, v, &c_s, &li_lum);
            if (cdf && P->collect) {
              /* guide learning: incident radiance / multi-sample density of the
               * indirect techniques, binned by direction */
              double dens = beta[ORC_T_BSDF] * pb + beta[ORC_T_GUIDED] * pg;
              if (dens > 0.0 && li_lum > 0.0)
                st->hist[(size_t)x->cell * ORC_GUIDE_BINS + guide_bin(wi)] += li_lum / dens;
            }
          }
        }
      }
      for (int c = 0; c < 3; ++c) Lr[c] += v[c] / beta[t];
      *cost += c_s;
      stat_add(R, x->cell, t, v, c_s, T);
    }
  }
}

int orc_render(const orc_scene_desc* scene, const orc_params* P, orc_state* st, int px_begin,
               int px_end) {
  if (!scene || !P || !st) return -1;
  if (!(P->techniques & 1)) return -1;
  if (P->max_depth < 1 || P->grid_n < 1) return -1;
  if (P->clamp_hi > 30.0 || P->clamp_lo < 0.0) return -1;
  if (P->mode == ORC_MODE_MARS && !P->has_estimate) return -2;
  if ((P->techniques & 4) && !st->guide_cdf) return -1;
  if ((P->techniques & 4) && (P->techniques & ORC_TECH_LIGHT)) return -1;
  if (P->max_depth + ORC_LIGHT_MAX + 2 > ORC_MAXP) return -1;
  ctx_t C;
  if (ctx_init(&C, scene, P) != 0) { ctx_free(&C); return -3; }
  if ((P->max_depth - 1) * C.bits > 64) { ctx_free(&C); return -1; }
  int npx = scene->width * scene->height;
  if (px_begin < 0 || px_end > npx || px_begin > px_end) { ctx_free(&C); return -1; }
  rnd_t R;
  R.C = &C;
  R.P = P;
  R.st = st;
  for (int t = 0; t < ORC_NT; ++t) R.on[t] = (P->techniques >> t) & 1;
  R.bd = (P->techniques & ORC_TECH_LIGHT) != 0;
  if (R.bd) R.on[ORC_T_LIGHT] = 1;
  for (int px = px_begin; px < px_end; ++px) {
    R.px = px;
    double u[4];
    rng4(P, (uint32_t)px, DIM_CAMERA, 0, u);
    int ix = px % scene->width, iy = px / scene->width;
    double sx = (2.0 * ((double)ix + u[0]) / scene->width - 1.0) * C.tanh * C.aspect;
    double sy = (1.0 - 2.0 * ((double)iy + u[1]) / scene->height) * C.tanh;
    v3 d = nrm(add(C.cam_f, add(scl(C.cam_r, sx), scl(C.cam_u, sy))));
    /* random walk (Sec. 3.1): W/p = 1 for the pinhole with box filter */
    ray_info ri;
    memset(&ri, 0, sizeof(ri));
    ri.camera = 1;
    ri.mult_child = 1.0f;
    ri.A = ri.S_ind = 1.0;
    for (int c = 0; c < 3; ++c) { ri.fcp[c] = 1.0; ri.T_child[c] = 1.0; }
    double v[3], cost;
    trace_sample(&R, C.cam_o, d, 1, 0, &ri, v, &cost, NULL);
    for (int c = 0; c < 3; ++c) st->image[3 * px + c] = v[c];
    st->counters[0] += cost;
    if (st->px_rays) st->px_rays[px] = cost;
  }
  ctx_free(&C);
  return 0;
}

/* ------------------------------------------------------------ test hooks
 * Brute-force checks of the light-side densities of the whole-path weights.
 * The renderer does not call these: they draw light subpath steps with the
 * renderer's own routines (emit_dir, light_bounce, closest_hit) and return the
 * density that the weights give the same steps (light_side_density), so that
 * a test can compare the frequency of the drawn landing points with it. */
static int debug_setup(ctx_t* C, const orc_scene_desc* scene, const orc_params* P, int l) {
  if (!scene || !P) return -1;
  if (ctx_init(C, scene, P) != 0) return -3;
  if (l < 0 || l >= C->n_lights) return -1;
  return 0;
}

int orc_debug_light_emit(const orc_scene_desc* scene, const orc_params* P, int l, const double* y0, int n,
                         const double* u, double* hit, int32_t* prim) {
  ctx_t C;
  int rc = debug_setup(&C, scene, P, l);
  if (rc != 0) { ctx_free(&C); return rc; }
  light_end e = light_end_at(&C, l, ld3(y0));
  v3 org = add(e.p, scl(e.n, C.eps));
  for (int i = 0; i < n; ++i) {
    hit_t h;
    v3 dir = emit_dir(e.n, u[2 * i], u[2 * i + 1]);
    prim[i] = closest_hit(&C, org, dir, &h) ? h.prim : -1;
    if (prim[i] >= 0) { hit[3 * i] = h.p.x; hit[3 * i + 1] = h.p.y; hit[3 * i + 2] = h.p.z; }
  }
  ctx_free(&C);
  return 0;
}

/* y_1: the first hit of the ray leaving light l's point y0 along d1 */
static int debug_first_vertex(const ctx_t* C, const light_end* e, const double* d1, hit_t* h1, v3* dir1) {
  *dir1 = nrm(ld3(d1));
  return closest_hit(C, add(e->p, scl(e->n, C->eps)), *dir1, h1);
}

int orc_debug_light_bounce(const orc_scene_desc* scene, const orc_params* P, int l, const double* y0,
                           const double* d1, int n, const double* u, double* hit, int32_t* prim) {
  ctx_t C;
  int rc = debug_setup(&C, scene, P, l);
  if (rc != 0) { ctx_free(&C); return rc; }
  light_end e = light_end_at(&C, l, ld3(y0));
  hit_t h1;
  v3 dir1;
  if (!debug_first_vertex(&C, &e, d1, &h1, &dir1)) { ctx_free(&C); return -4; }
  for (int i = 0; i < n; ++i) {
    double uu[4] = {u[3 * i], u[3 * i + 1], u[3 * i + 2], 0.0};
    v3 org, dir;
    double wb[3];
    hit_t h;
    prim[i] = -1;
    if (light_bounce(&C, &h1, scl(dir1, -1.0), uu, &org, &dir, wb) && closest_hit(&C, org, dir, &h)) {
      prim[i] = h.prim;
      hit[3 * i] = h.p.x; hit[3 * i + 1] = h.p.y; hit[3 * i + 2] = h.p.z;
    }
  }
  ctx_free(&C);
  return 0;
}

int orc_debug_light_density(const orc_scene_desc* scene, const orc_params* P, int l, const double* y0,
                            const double* d1, const double* x, double* out) {
  ctx_t C;
  int rc = debug_setup(&C, scene, P, l);
  if (rc != 0) { ctx_free(&C); return rc; }
  light_end e = light_end_at(&C, l, ld3(y0));
  hit_t h1, hx;
  v3 dir1;
  if (!debug_first_vertex(&C, &e, d1, &h1, &dir1)) { ctx_free(&C); return -4; }
  /* y_1 as a path vertex (camera order: dn towards the light point) */
  pathv_t z1;
  z1.p = h1.p;
  z1.ng = h1.ng;
  z1.mat = h1.mat;
  z1.dn = scl(dir1, -1.0);
  z1.tn = h1.t;
  z1.dp = mk(0, 0, 0);
  out[0] = light_side_density(&C, &z1, NULL, &e);
  /* x: the first hit of the ray from y_1 (offset as a bounce offsets it) towards x */
  v3 ns = dot(h1.ng, z1.dn) >= 0.0 ? h1.ng : scl(h1.ng, -1.0);
  v3 org = add(h1.p, scl(ns, C.eps));
  v3 dx = nrm(sub(ld3(x), org));
  out[1] = 0.0;
  if (closest_hit(&C, org, dx, &hx)) {
    pathv_t zx;
    zx.p = hx.p;
    zx.ng = hx.ng;
    zx.mat = hx.mat;
    zx.dn = scl(dx, -1.0);
    zx.tn = hx.t;
    zx.dp = mk(0, 0, 0);
    z1.dp = dx;
    out[1] = light_side_density(&C, &zx, &z1, &e);
  }
  ctx_free(&C);
  return 0;
}

/* ------------------------------------------------------------ image / update */
/* Brightness of a pixel for the rejection of the bidirectional application
 * (Sec. 5.1 "Implementation": the brightest pixels of a pass leave its image
 * variance estimate): luminance taken in float32, each product and sum rounded
 * in turn, so that the order of pixels equals the kernel's. */
static float bright_lum(const double* I) {
  float r = (float)I[0], g = (float)I[1], b = (float)I[2];
  float a = 0.2126f * r;
  float c = 0.7152f * g;
  float d = 0.0722f * b;
  float l = (a + c) + d;
  return l > 0.0f ? l : 0.0f;
}

double orc_image_stats(int W, int H, const double* img, double* run_sum, int n_prev,
                       double outlier, double* est_out) {
  return orc_image_stats_k(W, H, img, run_sum, n_prev, outlier, 0, est_out);
}

double orc_image_stats_k(int W, int H, const double* img, double* run_sum, int n_prev,
                         double outlier, int drop_k, double* est_out) {
  int n = W * H;
  double inv = 1.0 / (double)(n_prev + 1);
  double chmean[3] = {0, 0, 0};
  for (int p = 0; p < n; ++p)
    for (int c = 0; c < 3; ++c) {
      run_sum[3 * p + c] += img[3 * p + c];
      chmean[c] += run_sum[3 * p + c] * inv;
    }
  for (int c = 0; c < 3; ++c) chmean[c] /= (double)n;
  /* pixel estimate (reading; the paper denoises with OIDN, Sec. 4.1): 3x3 box
   * filter of the running mean over the in-image neighbours, floored */
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x)
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        int k = 0;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int xx = x + dx, yy = y + dy;
            if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
            s += run_sum[3 * (yy * W + xx) + c] * inv;
            k++;
          }
        double e = s / (double)k;
        double fl = 1e-3 * chmean[c];
        if (e < fl) e = fl;
        if (e < 1e-8) e = 1e-8;
        est_out[3 * (y * W + x) + c] = e;
      }
  /* image relative variance (Sec. 4.1 "Image estimates") with the sample
   * clamped at outlier x estimate ("Outlier clamping"); one sample per pixel */
  if (drop_k <= 0) {
    double vi = 0.0;
    for (int p = 0; p < n; ++p)
      for (int c = 0; c < 3; ++c) {
        double e = est_out[3 * p + c];
        double I = img[3 * p + c];
        if (I > outlier * e) I = outlier * e;
        double r = (I - e) / e;
        vi += r * r;
      }
    return vi / (3.0 * (double)n);
  }
  /* the bidirectional application's rejection instead (Sec. 5.1
   * "Implementation"): the drop_k brightest pixels (ties: lower index first)
   * leave the mean, the others enter unclamped */
  unsigned char* dropped = (unsigned char*)calloc((size_t)n, 1);
  for (int k = 0; k < drop_k && k < n; ++k) {
    int best = -1;
    float bl = -1.0f;
    for (int p = 0; p < n; ++p) {
      if (dropped[p]) continue;
      float l = bright_lum(img + 3 * p);
      if (l > bl) { bl = l; best = p; }  /* strict: the lower index wins a tie */
    }
    dropped[best] = 1;
  }
  double vi = 0.0;
  int kept = 0;
  for (int p = 0; p < n; ++p) {
    if (dropped[p]) continue;
    ++kept;
    for (int c = 0; c < 3; ++c) {
      double e = est_out[3 * p + c];
      double r = (img[3 * p + c] - e) / e;
      vi += r * r;
    }
  }
  free(dropped);
  return vi / (3.0 * (double)kept);
}

/* Fixed-point step (Eq. optimalBeta in its spatial form, Sec. 3.1): the cache
 * stores per channel q^RR = sqrt(C_I / C_t * E[<L_r,t>^2] / V_I) and
 * q^S = sqrt(C_I / C_t * V[<L_r,t>] / V_I); the vertex multiplies by T / I_px.
 * Moments are the per-sample (primary) moments of Sec. 4.1 "Local estimates". */
void orc_update_counts(int n_cells, int techniques, const double* stats, double VI, double CI,
                       float* q_rr, float* q_s, uint8_t* valid) {
  if (!(VI > 1e-12)) return;
  for (int c = 0; c < n_cells; ++c)
    for (int t = 0; t < ORC_NT; ++t) {
      /* slot 2 holds the guided technique or the light connection */
      int on = t == 2 ? (techniques & (4 | ORC_TECH_LIGHT)) != 0 : (techniques >> t) & 1;
      if (!on) continue;
      const double* s = stats + ((size_t)c * ORC_NT + t) * ORC_NSTAT;
      double n = s[0];
      if (n < 2.0 || !(s[7] > 0.0)) continue;
      double Ct = s[7] / n;
      for (int ch = 0; ch < 3; ++ch) {
        double m1 = s[1 + ch] / n;
        double m2 = s[4 + ch] / n;
        double var = m2 - m1 * m1;
        if (var < 0.0) var = 0.0;
        q_rr[((size_t)c * ORC_NT + t) * 3 + ch] = (float)sqrt(CI / Ct * m2 / VI);
        q_s[((size_t)c * ORC_NT + t) * 3 + ch] = (float)sqrt(CI / Ct * var / VI);
      }
      valid[(size_t)c * ORC_NT + t] = 1;
    }
}

void orc_guide_update(int n_cells, const double* hist, float* cdf) {
  for (int c = 0; c < n_cells; ++c) {
    const double* h = hist + (size_t)c * ORC_GUIDE_BINS;
    double H = 0.0;
    for (int b = 0; b < ORC_GUIDE_BINS; ++b) H += h[b];
    double run = 0.0;
    for (int b = 0; b < ORC_GUIDE_BINS; ++b) {
      double p = H > 0.0 ? 0.9 * h[b] / H + 0.1 / ORC_GUIDE_BINS : 1.0 / ORC_GUIDE_BINS;
      run += p;
      cdf[(size_t)c * ORC_GUIDE_BINS + b] = (float)run;
    }
    cdf[(size_t)c * ORC_GUIDE_BINS + ORC_GUIDE_BINS - 1] = 1.0f;
  }
}
