// render.cu -- wavefront MARS path tracer.  Per depth wave d (rays in
// [base[d], base[d] + count[d]) of the tile's arena):
//
//   k_trace  (wave d)  closest hit of every ray (camera rays for d = 1)
//   k_shade  (wave d)  emission reached by the ray, weighted against NEE
//                      (multi-sample balance heuristic, Sec. 3.1); at a vertex
//                      x_d with d <= D-1 the sampling half of the secondary
//                      estimator: counts beta_t from the cache (T(x)/I_px x q,
//                      three cases, clamp; Sec. 3.1 "Optimization", Sec. 4.1),
//                      Alg. 1, NEE samples written as shadow rays, BSDF / guided
//                      children appended to wave d+1 (warp-aggregated
//                      allocation)
//   k_shadow (wave d)  one thread per NEE shadow ray: any hit zeroes the sample
//
// then deepest first
//
//   k_reverse (wave d) every ray's sample value
//                        <L_r,t> = f|cos|/p_t (Le w_dir + w_ind <L_r(child vertex)>)
//                      and cost (rays in its subtree, counting itself), the
//                      vertex's <L_r> = sum_t 1/beta_t sum_s <L_r,t> (Sec. 3.1
//                      "Secondary estimator"), and the local statistics of
//                      Sec. 4.1 "Local estimates" (per cell and technique: n,
//                      sum v, sum v^2, sum cost), pre-reduced over runs of equal
//                      cells in a warp before float64 atomics.
//
// A tile whose arena overflowed commits nothing.
#include "device.cuh"

namespace mars {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// software prefetch of one line into L2 (no register result, no wait)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// every wave kernel accepts blocks of up to MAX_WAVE_THREADS threads; the launch
// shape (threads per block, grid) is a per-cache setting (WaveLaunch)
constexpr int MAX_WAVE_THREADS = 256;

__device__ __forceinline__ float4 f4(f3 a, float w) { return make_float4(a.x, a.y, a.z, w); }
__device__ __forceinline__ f3 fmin3(f3 a, f3 b) { return mk3(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z)); }

// NEE density (solid angle at x) of reaching point y on light l along wi
__device__ __forceinline__ float nee_pdf(const DevScene& s, int l, f3 x, f3 y, f3 wi) {
  const float4 l1 = __ldg(s.lights + 5 * l + 1), l2 = __ldg(s.lights + 5 * l + 2), l3 = __ldg(s.lights + 5 * l + 3);
  const float cosl = -dot(xyz(l3), wi);
  if (cosl <= 0.0f) return 0.0f;
  const f3 dv = y - x;
  return l1.w * dot(dv, dv) / (l2.w * cosl);
}

// pinhole camera ray of pixel px with box-filter jitter (W/p = 1)
__device__ __forceinline__ void camera_ray(const DevScene& s, const Rng& rng, uint32_t px, f3& o, f3& dir) {
  const float4 u = rng.u4(px, DIM_CAMERA, 0);
  const int ix = (int)(px % (uint32_t)s.width), iy = (int)(px / (uint32_t)s.width);
  const float sx = (2.0f * ((float)ix + u.x) / (float)s.width - 1.0f) * s.tanh_half * s.aspect;
  const float sy = (1.0f - 2.0f * ((float)iy + u.y) / (float)s.height) * s.tanh_half;
  const f3 cf = mk3(s.cam_f[0], s.cam_f[1], s.cam_f[2]);
  const f3 cr = mk3(s.cam_r[0], s.cam_r[1], s.cam_r[2]);
  const f3 cu = mk3(s.cam_u[0], s.cam_u[1], s.cam_u[2]);
  dir = normalize(cf + (cr * sx + cu * sy));
  o = mk3(s.cam_o[0], s.cam_o[1], s.cam_o[2]);
}

// slots [base, base + n) of wave d, clamped to the arena
struct Wave {
  unsigned long long base, n;
};
__device__ __forceinline__ Wave wave_of(const DevCounters* ctr, const Arena& a, int d) {
  const unsigned long long base = ctr->base[d], cnt = ctr->count[d];
  return {base, cnt < a.cap - base ? cnt : a.cap - base};
}

// A warp's allocation from a shared counter: its slots are contiguous, in lane
// order: lane l owns [base + incl - n, base + incl).
struct WarpAlloc {
  unsigned long long base;  // first slot of the warp (relative to the counter's origin)
  int incl;                 // inclusive prefix of the counts up to this lane
  int total;                // slots of the whole warp
};

// inclusive warp scan of a per-lane count; returns (inclusive prefix, warp total)
__device__ __forceinline__ int2 warp_scan(int n, int lane) {
  int incl = n;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += y;
  }
  return make_int2(incl, __shfl_sync(FULL, incl, 31));
}

// lane owning item k of a warp block: the smallest l with incl[l] > k
__device__ __forceinline__ int owner_lane(const int* incl, int k) {
  int lo = 0, hi = 31;
#pragma unroll
  for (int it = 0; it < 5; ++it) {
    const int mid = (lo + hi) >> 1;
    if (incl[mid] > k) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// warp sum of a thread's traversal counters, one atomic per counter and warp
__device__ __forceinline__ void flush_work(TraceWork w, unsigned long long* dst, DevCounters* ctr) {
#ifdef MARS_CHECKED
  if (w.bad) atomicOr(&ctr->check_flags, w.bad);
#else
  (void)ctr;
#endif
  unsigned long long v[4] = {w.nodes, w.quads, w.spheres, w.tris};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], off);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (v[k]) atomicAdd(dst + k, v[k]);
  }
}

__global__ void k_tile_init(DevCounters* ctr, const IterArgs* __restrict__ itp) {
  const unsigned long long n0 = (unsigned long long)(itp->tile_end - itp->tile_begin);
  const int t = threadIdx.x;
  if (t < MAXD + 2) {
    ctr->base[t] = 0;
    ctr->count[t] = (t == 1) ? n0 : 0ull;
    ctr->sbase[t] = 0;
    ctr->scount[t] = 0;
    ctr->slcount[t] = 0;
    ctr->lbase[t] = 0;
    ctr->lcount[t] = 0;
    ctr->vcount[t] = 0;
  }
  if (t == 0) {
    ctr->overflow = 0;
    ctr->demand = n0;
  }
}

__global__ void k_tile_finish(DevCounters* ctr, unsigned int* tile_status, const IterArgs* __restrict__ itp, int D) {
  if (threadIdx.x != 0) return;
  const int slot = itp->tile_slot;
  unsigned long long dem = 0;
  for (int d = 1; d <= D; ++d) {
    const unsigned long long e = ctr->base[d] + ctr->count[d];
    dem = e > dem ? e : dem;
  }
  ctr->demand = dem;
  if (!ctr->overflow) {
    unsigned long long tot = 0, sh = 0, sl = 0, lc = 0, lv = 0;
    for (int d = 1; d <= D; ++d) {
      tot += ctr->count[d];
      sh += ctr->scount[d];
      sl += ctr->slcount[d];
      lc += ctr->lcount[d];
      lv += ctr->vcount[d];
      ctr->wave_total[d] += ctr->count[d];
    }
    ctr->entries += tot;
    ctr->shadow_entries += sh;
    ctr->shadow_traced += sl;
    ctr->light_entries += lc;
    ctr->light_vertex_entries += lv;
  }
  tile_status[slot] = ctr->overflow;
  if (ctr->overflow) ctr->any_overflow = 1;
}

// Totals of a second tile lane's counters into the first's (added, then
// cleared in the source, so that a later merge adds only what came after).
__global__ void k_merge_lanes(DevCounters* dst, DevCounters* src) {
  if (threadIdx.x != 0) return;
  dst->shadow_entries += src->shadow_entries;
  dst->shadow_traced += src->shadow_traced;
  dst->rays += src->rays;
  dst->vertices += src->vertices;
  dst->est_vertices += src->est_vertices;
  dst->entries += src->entries;
  dst->light_entries += src->light_entries;
  dst->light_vertex_entries += src->light_vertex_entries;
  dst->light_rays += src->light_rays;
  dst->conn_rays += src->conn_rays;
  src->shadow_entries = src->shadow_traced = src->rays = src->vertices = src->est_vertices = src->entries = 0;
  src->light_entries = src->light_vertex_entries = src->light_rays = src->conn_rays = 0;
  for (int d = 0; d < MAXD + 2; ++d) {
    dst->wave_total[d] += src->wave_total[d];
    src->wave_total[d] = 0;
  }
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 4; ++q) {
      dst->trace_work[k][q] += src->trace_work[k][q];
      src->trace_work[k][q] = 0;
    }
  for (int t = 0; t < NT; ++t) {
    dst->sum_beta[t] += src->sum_beta[t];
    src->sum_beta[t] = 0.0;
  }
  if (src->any_overflow) dst->any_overflow = 1;
  src->any_overflow = 0;
  dst->check_flags |= src->check_flags;
  src->check_flags = 0;
  if (src->demand > dst->demand) dst->demand = src->demand;
}

// ------------------------------------------------------------------ trace
template <int MINB>
__global__ void __launch_bounds__(MAX_WAVE_THREADS, MINB) k_trace(const DevScene s, const DevCache c, const Arena a,
                                                         const IterArgs* __restrict__ itp, const int d) {
  const IterArgs it = *itp;
  const DevCounters* ctr = c.ctr;
  // after an overflow some slots of this wave were never written: stop, the
  // tile is re-rendered in smaller pieces
  if (ctr->overflow) return;
  const Wave w = wave_of(ctr, a, d);
  const Rng rng{it.seed, it.job, it.iteration};
  TraceWork tw;
  // One ray per thread, grid-stride.  (A persistent variant that refills the
  // lanes of finished rays from a warp-private pool measured 1.7x slower: the
  // refill bookkeeping costs more than the idle lanes it recovers.)
  for (unsigned long long li = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; li < w.n;
       li += gridDim.x * (unsigned long long)blockDim.x) {
    const unsigned long long i = w.base + li;
    if (!chk(i < a.cap, MARS_CHECK_ARENA, c.ctr)) break;
    f3 o, dir;
    bool alive = true;
    if (d == 1) {
      camera_ray(s, rng, (uint32_t)(it.tile_begin + li), o, dir);
    } else {
      const float4 r0 = a.R[0][i], r1 = a.R[1][i];
      o = xyz(r0);
      dir = xyz(r1);
      alive = r1.w > 0.0f;  // A = beta_t p_t is 0 for a drawn sample that is not traced
    }
    float t = 0.0f;
    int prim = -2;  // -2: not traced, -1: traced and missed
    // binary traversal: measured faster for closest hits than the 4-wide one,
    // whose per-node ordering and eager leaf tests cost more than the halved
    // node visits save; shadow rays use the 4-wide BVH
    if (alive) prim = trace_closest(s, o, dir, t, tw);
    a.H[i] = make_float2(t, __int_as_float(prim));
  }
  flush_work(tw, c.ctr->trace_work[0], c.ctr);
}

// ------------------------------------------------------------------ shade
// Per-warp staging area of k_shade: the context of the 32 vertices of a chunk,
// structure of arrays [field][lane], read by the lanes that draw their samples.
// C_Y and C_GP are used with light connections only (see k_shade<., true>).
enum {
  C_XO = 0, C_NS = 3, C_WO = 6, C_MTYPE = 9, C_ALPHA = 10, C_COL = 11, C_CELL = 14, C_PX = 15, C_LIN = 16,
  C_T = 18, C_B0 = 21, C_B1 = 22, C_B2 = 23, C_G0 = 24, C_MULT = 25, C_Y = 26, C_GP = 31, C_FIELDS = 32
};
struct ShadeWarpCtx {
  float f[C_FIELDS][32];
  int incl_ext[32];
  int incl_sh[32];
  int incl_lc[32];
};

// Whole-path weights with light connections (the bidirectional application,
// Sec. 5): the balance heuristic over every strategy of a full path z_1..z_n
// (z_n on a light) -- the camera path, NEE at z_{n-1}, light connection at
// z_i (i <= n - 2, n - 1 - i <= LIGHT_MAX light vertices) -- each strategy's
// density times its expected sample count.  Relative to the camera prefix
// C_k = prod_{j<k} bw_B(x_j) P->_j (P->_j: area density of x_{j+1} by BSDF
// sampling at x_j) the strategies that split the path before x_k add up to the
// window Y_k[l] = bw_L(x_{k-l}) prod_{m=k-l+1}^{k-2} P<-_m / prod_{m=k-l}^{k-1}
// bw_B P->_m (P<-_m: area density of x_m on a light subpath), which a ray
// carries forward as Z (Y of its parent times the parent's P<- towards the
// grandparent, Z[1] = the parent's light connection count) and the hit divides
// by the last step's bw_B P->.  The term of a light connection l vertices back
// at x_k is W_k[l] = Y_k[1] for l = 1 and Y_k[l] P<-_{k-1} for l >= 2 (P<-_{k-1}
// depends on the direction x_k continues in); a child carries Z[l] = W[l - 1].
// Emission hit at x_n from x_{n-1}:
//   w = bw_B P->_{n-1} / (bw_B P->_{n-1} + bw_N(x_{n-1}) pN + pN P<-_{n-1} sum_{l>=2} Z[l]);
// NEE at x_k towards y: w = bw_N pN / (bw_N pN + bw_B P->_k + pN P<-_k sum_l W_k[l]);
// light connections: the light kernel (bdpt.cu).
template <int MINB, bool BD>
__global__ void __launch_bounds__(MAX_WAVE_THREADS, MINB) k_shade(const DevScene s, const DevCache c, const Arena a,
                                                         const IterArgs* __restrict__ itp, const int d) {
  const IterArgs it = *itp;
  DevCounters* ctr = c.ctr;
  // block-level allocation below synchronises the block: decide the early exit
  // once per block (other blocks may raise the overflow flag meanwhile)
  __shared__ unsigned int blk_exit;
  __shared__ int blk_n[3][MAX_WAVE_THREADS / 32];
  __shared__ unsigned long long blk_base[3][MAX_WAVE_THREADS / 32];
  if (threadIdx.x == 0) blk_exit = ctr->overflow;
  __syncthreads();
  if (blk_exit) return;
  const Wave w = wave_of(ctr, a, d);
  const unsigned long long cnt = ctr->count[d];
  const unsigned long long base_next = w.base + cnt < a.cap ? w.base + cnt : a.cap;
  const unsigned long long sbase = d == 1 ? 0ull : ctr->sbase[d - 1] + ctr->scount[d - 1];
  const unsigned long long lbase = d == 1 ? 0ull : ctr->lbase[d - 1] + ctr->lcount[d - 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr->base[d + 1] = base_next;
    ctr->sbase[d] = sbase;
    if (BD) ctr->lbase[d] = lbase;
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int D = c.max_depth;
  const bool est_depth = d <= D - 1;
  const bool camera = d == 1;
  const bool on_b = c.techniques & MARS_TECH_BSDF, on_n = c.techniques & MARS_TECH_NEE,
             on_g = !BD && (c.techniques & MARS_TECH_GUIDED);
  // light connections are drawn at vertices of depth <= D - 2
  const bool on_l = BD && d <= D - 2;
  const Rng rng{it.seed, it.job, it.iteration};
  const float inf = __int_as_float(0x7f800000);
  extern __shared__ ShadeWarpCtx shade_ctx[];
  ShadeWarpCtx* ctx = shade_ctx + (threadIdx.x >> 5);

  // block-sized chunks (uniform trip count over the block); warp k of the block
  // takes the k-th 32 slots of the chunk
  for (unsigned long long b0 = blockIdx.x * (unsigned long long)blockDim.x; b0 < w.n;
       b0 += gridDim.x * (unsigned long long)blockDim.x) {
    const unsigned long long li = b0 + threadIdx.x;
    const bool active = li < w.n && chk(w.base + li < a.cap, MARS_CHECK_ARENA, ctr);
    const unsigned long long i = w.base + li;
    if (d > 1) {
      // the ray record of this thread's next slot, fetched into L2 meanwhile
      const unsigned long long ln = li + gridDim.x * (unsigned long long)blockDim.x;
      if (ln < w.n) {
        const unsigned long long in = w.base + ln;
#pragma unroll
        for (int k = 0; k < NR; ++k) prefetch_l2(a.R[k] + in);
      }
    }

    // ---- the ray of this slot and its hit
    f3 o = mk3(0.f, 0.f, 0.f), dir = mk3(0.f, 0.f, 1.f), T = mk3(1.f, 1.f, 1.f), fcp = mk3(1.f, 1.f, 1.f);
    float A = 1.0f, S_ind = 1.0f, bwN = 0.0f, invSb = 0.0f;
    uint64_t lin = 0;
    uint32_t px = 0, parent_cell = 0;
    float th = 0.0f, mult = 1.0f;
    int prim = -2;
    float Z[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // light connections: whole-path weight window
    if (active) {
      if (camera) {
        px = (uint32_t)(it.tile_begin + li);
        camera_ray(s, rng, px, o, dir);
      } else {
        mult = a.M[i];
        const float4 r0 = a.R[0][i], r1 = a.R[1][i], r2 = a.R[2][i], r3 = a.R[3][i], r4 = a.R[4][i];
        o = xyz(r0);
        px = __float_as_uint(r0.w);
        dir = xyz(r1);
        A = r1.w;
        T = xyz(r2);
        S_ind = r2.w;   // light connections: |cos| at the parent
        fcp = xyz(r3);
        bwN = r3.w;
        lin = (uint64_t)__float_as_uint(r4.x) | ((uint64_t)__float_as_uint(r4.y) << 32);
        if (BD) {
          const float4 r5 = a.R5[i];
          Z[0] = r4.z; Z[1] = r4.w; Z[2] = r5.x; Z[3] = r5.y; Z[4] = r5.z; Z[5] = r5.w;
        } else {
          parent_cell = __float_as_uint(r4.z);
          invSb = r4.w;
        }
      }
      const float2 h = a.H[i];
      th = h.x;
      prim = __float_as_int(h.y);
    }

    f3 E = mk3(0.f, 0.f, 0.f);
    float Le_lum = 0.0f;
    const f3 G = camera ? mk3(1.f, 1.f, 1.f)
                        : (BD ? fcp : (S_ind > 0.0f ? fcp * (A / S_ind) : mk3(0.f, 0.f, 0.f)));
    uint32_t flags = prim >= -1 ? F_TRACED : 0u;
    int gam[NT] = {0, 0, 0};
    float beta[NT] = {0.f, 0.f, 0.f};
    float Y[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // light connections: Y_k[1..5]
    float gprev = 0.0f;                        // |cos| at the parent / t^2
    int cell = 0;
    f3 p = mk3(0.f, 0.f, 0.f), ns = mk3(0.f, 0.f, 1.f), wo = mk3(0.f, 0.f, 1.f);
    f3 climit = mk3(inf, inf, inf);
    Mat mat;
    mat.type = 0;
    mat.alpha = 1.0f;
    mat.col = mk3(0.f, 0.f, 0.f);
    if (prim >= 0 && chk(prim < s.n_prims, MARS_CHECK_PRIM, ctr)) {
      p = o + dir * th;
      const f3 ng = prim_normal(s.prims, prim, p);
      wo = dir * -1.0f;
      int m = prim_material(s.prims, prim);
      if (!chk(m >= 0 && m < s.n_mats, MARS_CHECK_MATERIAL, ctr)) m = 0;
      const float4 m0 = __ldg(s.mats + 3 * m), m1 = __ldg(s.mats + 3 * m + 1), m2 = __ldg(s.mats + 3 * m + 2);
      const float cosg = dot(ng, wo);
      // the last step's bw_B P-> (area density of this hit from the parent)
      const float inv_t2 = 1.0f / (th * th);
      const float cp_prev = BD && !camera ? A * fabsf(cosg) * inv_t2 : 0.0f;
      if (cosg > 0.0f && m0.w > 0.0f) {
        float w_dir = 1.0f;
        if (!camera && BD) {
          float sz = Z[1] + Z[2] + Z[3] + Z[4] + Z[5];
          float pN = 0.0f;
          if (prim < s.n_quads) {
            const int l = __float_as_int(__ldg(&s.prims[4 * prim + 3].w));
            if (l >= 0 && chk(l < s.n_lights, MARS_CHECK_LIGHT, ctr))
              pN = __ldg(&s.lights[5 * l + 1].w) / __ldg(&s.lights[5 * l + 2].w);
          }
          const float lpe = cosg * INV_PI_F * S_ind * inv_t2;   // P<-_{n-1}: cosine emission towards the parent
          const float den = cp_prev + bwN * pN + pN * lpe * sz;
          w_dir = den > 0.0f ? cp_prev / den : 0.0f;
        } else if (!camera) {
          float pn = 0.0f;
          if (bwN > 0.0f && prim < s.n_quads) {
            const int l = __float_as_int(__ldg(&s.prims[4 * prim + 3].w));
            if (l >= 0) pn = nee_pdf(s, l, o, p, dir);
          }
          const float den = S_ind + bwN * pn;
          w_dir = den > 0.0f ? A / den : 0.0f;
        }
        const f3 Le = xyz(m2);
        E = mul(fcp, Le * w_dir);
        Le_lum = lum(Le);
      }
      if (est_depth && m0.z > 0.0f) {
        // ---- budgets and Alg. 1 at vertex x_d
        flags |= F_EST;
        ns = cosg >= 0.0f ? ng : ng * -1.0f;
        cell = c.oct_nodes ? octree_cell(s, c.oct_nodes, p) : cell_of(s, c.grid_n, p);
        if (!chk(cell >= 0 && cell < c.n_cells, MARS_CHECK_CELL, ctr)) cell = 0;
        if (!chk(px < (uint32_t)c.n_pixels, MARS_CHECK_PIXEL, ctr)) px = 0;
        mat.type = (int)m0.x;
        mat.alpha = m0.y;
        mat.col = xyz(m1);
        const float4 est = it.has_estimate ? c.est[px] : make_float4(1.f, 1.f, 1.f, 0.f);
        if (!BD && it.collect && it.has_estimate) {
          climit.x = T.x > 0.0f ? it.outlier * est.x / T.x : inf;
          climit.y = T.y > 0.0f ? it.outlier * est.y / T.y : inf;
          climit.z = T.z > 0.0f ? it.outlier * est.z / T.z : inf;
        }
        // counts without learned statistics: one NEE (and light connection)
        // sample and one continuation sample split evenly over BSDF and guided
        // sampling
        const float base_cont = (on_b && on_g) ? 0.5f : 1.0f;
        const unsigned on_mask = (on_b ? 1u : 0u) | (on_n ? 2u : 0u) | ((on_g || on_l) ? 4u : 0u);
        vertex_budgets(c, it, cell, T, est, mult, on_mask, base_cont, BD ? 1.0f : base_cont, beta);
        if (BD && !camera) {
          const float icp = cp_prev > 0.0f ? 1.0f / cp_prev : 0.0f;
#pragma unroll
          for (int l = 0; l < 5; ++l) Y[l] = Z[l] * icp;
          gprev = S_ind * inv_t2;
        }
        // Alg. 1: one uniform decides the rounding of every technique
        float r = rng.u4(px, DIM_ROUND, lin).x;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          if (!((on_mask >> t) & 1u)) continue;
          const float sm = beta[t] + r;
          const int g = (int)floorf(sm);
          gam[t] = g;
          r = sm - (float)g;
        }
      }
    }

    // ---- slots for the children (wave d+1), the NEE shadow rays and the light
    // connection samples: warp scans, then one atomic per counter and block
    // (every block of the grid allocates from the same counters)
    const int n_ext = BD ? gam[0] : gam[0] + gam[2], n_sh = gam[1], n_lc = BD ? gam[2] : 0;
    const int2 se = warp_scan(n_ext, lane), ss = warp_scan(n_sh, lane);
    const int2 sl = BD ? warp_scan(n_lc, lane) : make_int2(0, 0);
    if (lane == 31) {
      blk_n[0][warp] = se.y;
      blk_n[1][warp] = ss.y;
      blk_n[2][warp] = sl.y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int te = 0, ts = 0, tl = 0;
      for (int k = 0; k < nwarps; ++k) {
        const int e = blk_n[0][k], h = blk_n[1][k], q = blk_n[2][k];
        blk_n[0][k] = te;
        blk_n[1][k] = ts;
        blk_n[2][k] = tl;
        te += e;
        ts += h;
        tl += q;
      }
      const unsigned long long be = te > 0 ? atomicAdd(&ctr->count[d + 1], (unsigned long long)te) : 0ull;
      const unsigned long long bs = ts > 0 ? atomicAdd(&ctr->scount[d], (unsigned long long)ts) : 0ull;
      const unsigned long long bl = (BD && tl > 0) ? atomicAdd(&ctr->lcount[d], (unsigned long long)tl) : 0ull;
      for (int k = 0; k < nwarps; ++k) {
        blk_base[0][k] = be + (unsigned long long)blk_n[0][k];
        blk_base[1][k] = bs + (unsigned long long)blk_n[1][k];
        blk_base[2][k] = bl + (unsigned long long)blk_n[2][k];
      }
    }
    __syncthreads();
    const WarpAlloc ae{blk_base[0][warp], se.x, se.y};
    const WarpAlloc as{blk_base[1][warp], ss.x, ss.y};
    const WarpAlloc al{blk_base[2][warp], sl.x, sl.y};
    const unsigned long long first = base_next + ae.base + (unsigned long long)(ae.incl - n_ext);
    const unsigned long long sfirst = sbase + as.base + (unsigned long long)(as.incl - n_sh);
    const unsigned long long lfirst = lbase + al.base + (unsigned long long)(al.incl - n_lc);
    const bool fits = first + (unsigned long long)n_ext <= a.cap && sfirst + (unsigned long long)n_sh <= a.scap &&
                      (!BD || lfirst + (unsigned long long)n_lc <= a.lcap);
    if ((n_ext > 0 || n_sh > 0 || n_lc > 0) && !fits) atomicOr(&ctr->overflow, 1u);

    // ---- vertex record of this slot
    if (active) {
      flags |= (uint32_t)gam[0] | ((uint32_t)gam[1] << 8) | ((uint32_t)gam[2] << 16);
      a.V[0][i] = f4(E, __uint_as_float(flags));
      if (flags & F_EST) {
        a.V[1][i] = f4(G, 0.0f);
        a.V[2][i] = f4(climit, __uint_as_float((uint32_t)cell));
        a.V[3][i] = make_float4(beta[0], beta[1], beta[2], __uint_as_float((uint32_t)(fits && BD ? lfirst : 0ull)));
        // the hit record is dead from here on: keep the first child and first
        // shadow-ray slots in it for the reverse pass
        a.H[i] = make_float2(__uint_as_float((uint32_t)(fits ? first : 0ull)),
                             __uint_as_float((uint32_t)(fits ? sfirst : 0ull)));
      }
      if (on_g && it.collect && !camera && (flags & F_TRACED))
        a.V[4][i] = make_float4(Le_lum, invSb, __uint_as_float(parent_cell), __int_as_float(guide_bin(dir)));
    }
    if (ae.total == 0 && as.total == 0 && al.total == 0) continue;  // warp-uniform; no block barrier follows

    // ---- stage the vertex context of every lane for the cooperative loops
    {
      const Frame fr = make_frame(ns);
      const f3 wol = fr.to_local(wo);
      const f3 xo = p + ns * s.eps;
      float* cx = ctx->f[0];
      cx[C_XO * 32 + lane] = xo.x; cx[(C_XO + 1) * 32 + lane] = xo.y; cx[(C_XO + 2) * 32 + lane] = xo.z;
      cx[C_NS * 32 + lane] = ns.x; cx[(C_NS + 1) * 32 + lane] = ns.y; cx[(C_NS + 2) * 32 + lane] = ns.z;
      cx[C_WO * 32 + lane] = wol.x; cx[(C_WO + 1) * 32 + lane] = wol.y; cx[(C_WO + 2) * 32 + lane] = wol.z;
      cx[C_MTYPE * 32 + lane] = __int_as_float(mat.type);
      cx[C_ALPHA * 32 + lane] = mat.alpha;
      cx[C_COL * 32 + lane] = mat.col.x; cx[(C_COL + 1) * 32 + lane] = mat.col.y; cx[(C_COL + 2) * 32 + lane] = mat.col.z;
      cx[C_CELL * 32 + lane] = __int_as_float(cell);
      cx[C_PX * 32 + lane] = __uint_as_float(px);
      cx[C_LIN * 32 + lane] = __uint_as_float((uint32_t)lin);
      cx[(C_LIN + 1) * 32 + lane] = __uint_as_float((uint32_t)(lin >> 32));
      cx[C_T * 32 + lane] = T.x; cx[(C_T + 1) * 32 + lane] = T.y; cx[(C_T + 2) * 32 + lane] = T.z;
      cx[C_B0 * 32 + lane] = beta[0];
      cx[C_B1 * 32 + lane] = beta[1];
      cx[C_B2 * 32 + lane] = beta[2];
      cx[C_G0 * 32 + lane] = __int_as_float(gam[0]);
      cx[C_MULT * 32 + lane] = mult;
      if (BD) {
#pragma unroll
        for (int l = 0; l < 5; ++l) cx[(C_Y + l) * 32 + lane] = Y[l];
        cx[C_GP * 32 + lane] = gprev;
      }
      ctx->incl_ext[lane] = ae.incl;
      ctx->incl_sh[lane] = as.incl;
      ctx->incl_lc[lane] = al.incl;
    }
    __syncwarp();
    const float* cx = ctx->f[0];

    // NEE samples (primary estimators of NEE), one per lane and pass; the value
    // assumes the light is visible (the shadow kernel zeroes it otherwise)
    for (int k0 = 0; k0 < as.total; k0 += 32) {
      const int k = k0 + lane;
      const unsigned long long j = sbase + as.base + (unsigned long long)k;
      bool trace = false;
      f3 xo = mk3(0.f, 0.f, 0.f), wi = mk3(0.f, 0.f, 1.f);
      float tmax = -1.0f;
      if (k < as.total && j < a.scap) {
        const int L = owner_lane(ctx->incl_sh, k);
        const int sidx = k - (L > 0 ? ctx->incl_sh[L - 1] : 0);
        xo = mk3(cx[C_XO * 32 + L], cx[(C_XO + 1) * 32 + L], cx[(C_XO + 2) * 32 + L]);
        const f3 vns = mk3(cx[C_NS * 32 + L], cx[(C_NS + 1) * 32 + L], cx[(C_NS + 2) * 32 + L]);
        const f3 wol = mk3(cx[C_WO * 32 + L], cx[(C_WO + 1) * 32 + L], cx[(C_WO + 2) * 32 + L]);
        Mat m;
        m.type = __float_as_int(cx[C_MTYPE * 32 + L]);
        m.alpha = cx[C_ALPHA * 32 + L];
        m.col = mk3(cx[C_COL * 32 + L], cx[(C_COL + 1) * 32 + L], cx[(C_COL + 2) * 32 + L]);
        const uint32_t vpx = __float_as_uint(cx[C_PX * 32 + L]);
        const uint64_t vlin = (uint64_t)__float_as_uint(cx[C_LIN * 32 + L]) |
                              ((uint64_t)__float_as_uint(cx[(C_LIN + 1) * 32 + L]) << 32);
        const float bB = cx[C_B0 * 32 + L], bN = cx[C_B1 * 32 + L], bG = cx[C_B2 * 32 + L];
        const float bwB = on_b ? (it.aware ? bB : 1.0f) : 0.0f;
        const float bwNv = on_n ? (it.aware ? bN : 1.0f) : 0.0f;
        const float bwG = on_g ? (it.aware ? bG : 1.0f) : 0.0f;
        const float4 u = rng.u4(vpx, 32u + (uint32_t)sidx, vlin);
        int l = s.n_lights - 1;
        for (int q = 0; q < s.n_lights; ++q)
          if (u.x < __ldg(&s.lights[5 * q].w)) { l = q; break; }
        const float4 l0 = __ldg(s.lights + 5 * l), l1 = __ldg(s.lights + 5 * l + 1),
                     l2 = __ldg(s.lights + 5 * l + 2), l4 = __ldg(s.lights + 5 * l + 4);
        const f3 y = xyz(l0) + (xyz(l1) * u.y + xyz(l2) * u.z);
        const f3 dv = y - xo;
        const float dist = sqrtf(dot(dv, dv));
        wi = dv * (1.0f / dist);
        const float pn = nee_pdf(s, l, xo, y, wi);
        const float ci = dot(vns, wi);
        f3 v = mk3(0.f, 0.f, 0.f);
        if (pn > 0.0f && ci > 0.0f) {
          const Frame fr = make_frame(vns);
          float pb;
          const f3 wil = fr.to_local(wi);
          const f3 fc = bsdf_eval(m, wol, wil, pb);
          const float pg = on_g ? guide_pdf(c.guide_cdf + (size_t)__float_as_int(cx[C_CELL * 32 + L]) * GUIDE_BINS, wi)
                                : 0.0f;
          if (nonzero(fc)) {
            if (BD) {
              // the full path x_1..x_d, y: weight over every strategy
              const float4 l3 = __ldg(s.lights + 5 * l + 3);
              const float pN = l1.w / l2.w;
              const float cosl = -dot(xyz(l3), wi);
              const float id2 = 1.0f / (dist * dist);
              const float t_nee = bwNv * pN;
              const float t_cam = bwB * pb * cosl * id2;
              // light connections l vertices back: W[1] = Y[1], W[l] = Y[l] P<-_{d-1} (l >= 2)
              const float y1 = cx[C_Y * 32 + L];
              float sy = 0.0f;
#pragma unroll
              for (int q = 1; q < 5; ++q) sy += cx[(C_Y + q) * 32 + L];
              float t_lc = 0.0f;
              if (y1 > 0.0f || sy > 0.0f) {
                float lp = 0.0f;
                if (sy > 0.0f) {
                  float prev;
                  const f3 frev = bsdf_eval(m, wil, wol, prev);   // at x_d, light arriving along wi
                  const float qx = prev > 0.0f ? fminf(1.0f, max_channel(frev) / prev) : 0.0f;
                  lp = prev * qx * cx[C_GP * 32 + L];
                }
                t_lc = pN * (cosl * INV_PI_F * ci * id2) * (y1 + lp * sy);
              }
              const float den = t_nee + t_cam + t_lc;
              const float sc = den > 0.0f ? t_nee / (den * pn) : 0.0f;
              v = mk3(fc.x * l4.x * sc, fc.y * l4.y * sc, fc.z * l4.z * sc);
            } else {
              // f|cos| Le / p_N times the balance weight beta_N p_N / den: p_N cancels
              const float den = bwB * pb + bwG * pg + bwNv * pn;
              const float sc = bwNv / den;
              v = mk3(fc.x * l4.x * sc, fc.y * l4.y * sc, fc.z * l4.z * sc);
            }
          }
        }
        a.SH[2][j] = f4(v, 0.0f);
        // a sample of value 0 needs no shadow ray
        trace = nonzero(v);
        tmax = dist - s.eps;
      }
      // compacted list of the shadow rays to trace: one atomic per warp
      const unsigned need = __ballot_sync(FULL, trace);
      if (need) {
        unsigned long long lb = 0;
        if (lane == 0) lb = atomicAdd(&ctr->slcount[d], (unsigned long long)__popc(need));
        lb = __shfl_sync(FULL, lb, 0);
        if (trace) {
          const unsigned long long pos = sbase + lb + (unsigned long long)__popc(need & ((1u << lane) - 1u));
          if (pos < a.scap) {
            a.SL[pos] = (unsigned int)j;
            a.SH[0][j] = f4(xo, tmax);
            a.SH[1][j] = f4(wi, 0.0f);
          }
        }
      }
    }

    // BSDF and guided children (primary estimators that continue the path);
    // a vertex's BSDF children come first, then its guided children
    for (int k0 = 0; k0 < ae.total; k0 += 32) {
      const int k = k0 + lane;
      const unsigned long long j = base_next + ae.base + (unsigned long long)k;
      if (k < ae.total && j < a.cap) {
        const int L = owner_lane(ctx->incl_ext, k);
        const int kk = k - (L > 0 ? ctx->incl_ext[L - 1] : 0);
        const int g0 = __float_as_int(cx[C_G0 * 32 + L]);
        const int t = kk < g0 ? 0 : 2;
        const int sidx = t == 0 ? kk : kk - g0;
        const f3 xo = mk3(cx[C_XO * 32 + L], cx[(C_XO + 1) * 32 + L], cx[(C_XO + 2) * 32 + L]);
        const f3 vns = mk3(cx[C_NS * 32 + L], cx[(C_NS + 1) * 32 + L], cx[(C_NS + 2) * 32 + L]);
        const f3 wol = mk3(cx[C_WO * 32 + L], cx[(C_WO + 1) * 32 + L], cx[(C_WO + 2) * 32 + L]);
        Mat m;
        m.type = __float_as_int(cx[C_MTYPE * 32 + L]);
        m.alpha = cx[C_ALPHA * 32 + L];
        m.col = mk3(cx[C_COL * 32 + L], cx[(C_COL + 1) * 32 + L], cx[(C_COL + 2) * 32 + L]);
        const int vcell = __float_as_int(cx[C_CELL * 32 + L]);
        const uint32_t vpx = __float_as_uint(cx[C_PX * 32 + L]);
        const uint64_t vlin = (uint64_t)__float_as_uint(cx[C_LIN * 32 + L]) |
                              ((uint64_t)__float_as_uint(cx[(C_LIN + 1) * 32 + L]) << 32);
        const f3 vT = mk3(cx[C_T * 32 + L], cx[(C_T + 1) * 32 + L], cx[(C_T + 2) * 32 + L]);
        const float bB = cx[C_B0 * 32 + L], bN = cx[C_B1 * 32 + L], bG = cx[C_B2 * 32 + L];
        const float bwB = on_b ? (it.aware ? bB : 1.0f) : 0.0f;
        const float bwNv = on_n ? (it.aware ? bN : 1.0f) : 0.0f;
        const float bwG = on_g ? (it.aware ? bG : 1.0f) : 0.0f;
        const float bt = t == 0 ? bB : bG;
        const float* cdf = on_g ? c.guide_cdf + (size_t)vcell * GUIDE_BINS : nullptr;
        const Frame fr = make_frame(vns);
        const float4 u = rng.u4(vpx, (uint32_t)(t * 32 + sidx), vlin);
        f3 wi = mk3(0.f, 0.f, 1.f);
        bool ok;
        float pt = 0.0f;
        if (t == 0) {
          f3 wl;
          ok = bsdf_sample(m, wol, u.x, u.y, wl);
          if (ok) wi = fr.to_world(wl);
        } else {
          int b = guide_pick(cdf, u.x);
          if (!chk(b >= 0 && b < GUIDE_BINS, MARS_CHECK_BIN, ctr)) b = 0;
          wi = guide_dir(b, u.y, u.z);
          pt = guide_bin_prob(cdf, b) * (GUIDE_BINS / (4.0f * PI_F));
          ok = dot(wi, vns) > 0.0f;
        }
        float cA = 0.0f, cS = 0.0f, cinvSb = 0.0f;
        f3 cf = mk3(0.f, 0.f, 0.f), cT = mk3(0.f, 0.f, 0.f);
        float cz[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ok) {
          float pb;
          const f3 wil = fr.to_local(wi);
          const f3 fc = bsdf_eval(m, wol, wil, pb);
          const float pg = on_g ? guide_pdf(cdf, wi) : 0.0f;
          if (t == 0) pt = pb;
          if (pt > 0.0f && nonzero(fc)) {
            const float ipt = 1.0f / pt;
            cf = mk3(fc.x * ipt, fc.y * ipt, fc.z * ipt);
            cA = (t == 0 ? bwB : bwG) * pt;
            if (BD) {
              // no MIS weight on the continuation; the ray carries |cos| here and
              // the whole-path window
              const float wb = 1.0f / bt;
              cT = mk3(vT.x * cf.x * wb, vT.y * cf.y * wb, vT.z * cf.z * wb);
              cS = dot(vns, wi);
              // Z of the child: Z[1] = bw_L here, Z[l] = W[l - 1] (W[1] = Y[1], W[l] = Y[l] P<-_{d-1})
              cz[0] = on_l ? (it.aware ? bG : 1.0f) : 0.0f;
              cz[1] = cx[C_Y * 32 + L];
              float sy = 0.0f;
#pragma unroll
              for (int q = 1; q < 5; ++q) sy += cx[(C_Y + q) * 32 + L];
              if (sy > 0.0f) {
                float prev;
                const f3 frev = bsdf_eval(m, wil, wol, prev);   // P<- of the parent towards its parent
                const float qx = prev > 0.0f ? fminf(1.0f, max_channel(frev) / prev) : 0.0f;
                const float lp = prev * qx * cx[C_GP * 32 + L];
#pragma unroll
                for (int q = 1; q < 5; ++q) cz[q + 1] = cx[(C_Y + q) * 32 + L] * lp;
              }
            } else {
              cS = bwB * pb + bwG * pg;
              const float w_ind = cA / cS;
              const float wb = w_ind / bt;
              cT = mk3(vT.x * cf.x * wb, vT.y * cf.y * wb, vT.z * cf.z * wb);
              const float sb = bB * pb + (on_g ? bG * pg : 0.0f);
              cinvSb = sb > 0.0f ? 1.0f / sb : 0.0f;
            }
          }
        }
        const uint64_t digit = (uint64_t)(t == 0 ? sidx + 1 : 32 + sidx + 1);
        const uint64_t clin = (vlin << c.bits) | digit;
        a.R[0][j] = f4(xo, __uint_as_float(vpx));
        a.R[1][j] = f4(wi, cA);
        a.R[2][j] = f4(cT, cS);
        a.R[3][j] = f4(cf, bwNv);
        if (BD) {
          a.R[4][j] = make_float4(__uint_as_float((uint32_t)clin), __uint_as_float((uint32_t)(clin >> 32)), cz[0], cz[1]);
          a.R5[j] = make_float4(cz[2], cz[3], cz[4], cz[5]);
        } else {
          a.R[4][j] = make_float4(__uint_as_float((uint32_t)clin), __uint_as_float((uint32_t)(clin >> 32)),
                                  __uint_as_float((uint32_t)vcell), cinvSb);
        }
        a.M[j] = cx[C_MULT * 32 + L] * bt;
      }
    }

    // light connection samples: the camera vertex's context for the light kernel
    if (BD) {
      for (int k0 = 0; k0 < al.total; k0 += 32) {
        const int k = k0 + lane;
        const unsigned long long j = lbase + al.base + (unsigned long long)k;
        if (k < al.total && j < a.lcap) {
          const int L = owner_lane(ctx->incl_lc, k);
          const int sidx = k - (L > 0 ? ctx->incl_lc[L - 1] : 0);
          const f3 vns = mk3(cx[C_NS * 32 + L], cx[(C_NS + 1) * 32 + L], cx[(C_NS + 2) * 32 + L]);
          const f3 wow = make_frame(vns).to_world(mk3(cx[C_WO * 32 + L], cx[(C_WO + 1) * 32 + L],
                                                      cx[(C_WO + 2) * 32 + L]));
          const float bB = cx[C_B0 * 32 + L], bN = cx[C_B1 * 32 + L], bL = cx[C_B2 * 32 + L];
          a.LJ[0][j] = make_float4(cx[C_XO * 32 + L], cx[(C_XO + 1) * 32 + L], cx[(C_XO + 2) * 32 + L],
                                   cx[C_PX * 32 + L]);
          a.LJ[1][j] = f4(vns, __uint_as_float((uint32_t)__float_as_int(cx[C_MTYPE * 32 + L]) |
                                               ((uint32_t)sidx << 8) | ((uint32_t)d << 16)));
          a.LJ[2][j] = make_float4(cx[C_COL * 32 + L], cx[(C_COL + 1) * 32 + L], cx[(C_COL + 2) * 32 + L],
                                   cx[C_ALPHA * 32 + L]);
          a.LJ[3][j] = f4(wow, cx[C_MULT * 32 + L]);
          a.LJ[4][j] = make_float4(cx[C_T * 32 + L], cx[(C_T + 1) * 32 + L], cx[(C_T + 2) * 32 + L], bB);
          a.LJ[5][j] = make_float4(it.aware ? bB : 1.0f, on_n ? (it.aware ? bN : 1.0f) : 0.0f,
                                   it.aware ? bL : 1.0f, cx[C_GP * 32 + L]);
          a.LJ[6][j] = make_float4(cx[C_Y * 32 + L], cx[(C_Y + 1) * 32 + L], cx[(C_Y + 2) * 32 + L],
                                   cx[(C_Y + 3) * 32 + L]);
          a.LJ[7][j] = make_float4(cx[C_LIN * 32 + L], cx[(C_LIN + 1) * 32 + L], 0.0f, 0.0f);
        }
      }
    }
    __syncwarp();  // the context is overwritten by the next chunk
  }
}

// ----------------------------------------------------------------- shadow
template <int MINB>
__global__ void __launch_bounds__(MAX_WAVE_THREADS, MINB) k_shadow(const DevScene s, const DevCache c, const Arena a,
                                                           const int d) {
  const DevCounters* ctr = c.ctr;
  if (ctr->overflow) return;
  // the listed shadow rays of wave d: SL[sbase, sbase + slcount), slot indices
  // into the wave's shadow region (at most scount of them)
  const unsigned long long sb = ctr->sbase[d], sl = ctr->slcount[d];
  const unsigned long long n = sl < a.scap - sb ? sl : a.scap - sb;
  TraceWork tw;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
       k += gridDim.x * (unsigned long long)blockDim.x) {
    const unsigned long long j = a.SL[sb + k];
    if (!chk(j < a.scap, MARS_CHECK_SHADOW, c.ctr)) continue;
    const float4 s0 = a.SH[0][j];
    if (!(s0.w > 0.0f)) continue;
    const float4 s1 = a.SH[1][j];
    if (trace_any4(s, xyz(s0), xyz(s1), s0.w, tw)) a.SH[2][j] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  flush_work(tw, c.ctr->trace_work[1], c.ctr);
}

// ---------------------------------------------------------------- reverse
// inclusive scan restricted to runs of equal keys (start = first lane of the run)
__device__ __forceinline__ float seg_scan(float v, int lane, int start) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float u = __shfl_up_sync(FULL, v, off);
    if (lane - off >= start) v += u;
  }
  return v;
}

template <int MINB, bool BD>
__global__ void __launch_bounds__(MAX_WAVE_THREADS, MINB) k_reverse(const DevScene s, const DevCache c, const Arena a,
                                                             const IterArgs* __restrict__ itp, const int d) {
  const IterArgs it = *itp;
  DevCounters* ctr = c.ctr;
  if (ctr->overflow) return;  // the tile is re-rendered; commit nothing
  const Wave w = wave_of(ctr, a, d);
  const int lane = threadIdx.x & 31;
  const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nw = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
  const bool on_n = c.techniques & MARS_TECH_NEE, on_g = !BD && (c.techniques & MARS_TECH_GUIDED);
  const bool collect = it.collect != 0;
  // iteration counters of this thread's slots: one warp reduction and one
  // atomic per counter and warp at the end, not per chunk (every warp of the
  // grid adds to the same few addresses)
  unsigned long long n_traced = 0, n_est = 0, n_rays = 0;
  double sb0 = 0.0, sb1 = 0.0, sb2 = 0.0;

  for (unsigned long long c0 = gw * 32; c0 < w.n; c0 += nw * 32) {
    const unsigned long long li = c0 + lane;
    const bool active = li < w.n && chk(w.base + li < a.cap, MARS_CHECK_ARENA, ctr);
    const unsigned long long i = w.base + li;
    {
      // the records of this thread's next slot, fetched into L2 while this one
      // is processed (the reverse pass reads them long after they were written)
      const unsigned long long ln = li + nw * 32;
      if (ln < w.n) {
        const unsigned long long in = w.base + ln;
        prefetch_l2(a.V[0] + in);
        prefetch_l2(a.H + in);
        prefetch_l2(a.V[1] + in);
        prefetch_l2(a.V[2] + in);
        prefetch_l2(a.V[3] + in);
      }
    }
    uint32_t flags = 0;
    f3 E = mk3(0.f, 0.f, 0.f), Lr = mk3(0.f, 0.f, 0.f);
    uint32_t csub = 0;
    uint32_t key = 0xffffffffu;
    float st[NT][NSTAT];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int k = 0; k < NSTAT; ++k) st[t][k] = 0.0f;
    float bt[NT] = {0.f, 0.f, 0.f};
    if (active) {
      // one round trip for the flags and the first child / shadow-ray slots,
      // then every other load of the vertex is issued before any is used
      const float4 v0 = a.V[0][i];
      const float2 fs = a.H[i];
      E = xyz(v0);
      flags = __float_as_uint(v0.w);
      const bool guide_dep = on_g && collect && d >= 2 && (flags & F_TRACED);
      float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (guide_dep) v4 = a.V[4][i];
      if (flags & F_EST) {
        int gB = flags & 0xff, gN = (flags >> 8) & 0xff, gG = (flags >> 16) & 0xff;
        // with light connections slot 2 holds the light connection samples,
        // which are not children
        int gL = BD ? gG : 0;
        if (BD) gG = 0;
        int ne = gB + gG;
        unsigned long long first = __float_as_uint(fs.x), sf = __float_as_uint(fs.y);
        // the children and NEE values lie inside the arena (else read none)
        const bool in_a = chk(first + (unsigned long long)ne <= a.cap, MARS_CHECK_ARENA, ctr);
        const bool in_s = chk(sf + (unsigned long long)gN <= a.scap, MARS_CHECK_SHADOW, ctr);
        if (!in_a) { first = 0; ne = 0; gB = 0; gG = 0; }
        if (!in_s) { sf = 0; gN = 0; }
        const float4 v1 = a.V[1][i], v2 = a.V[2][i], v3 = a.V[3][i];
        float4 pn[4], pe[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          pn[q] = q < gN ? a.SH[2][sf + q] : make_float4(0.f, 0.f, 0.f, 0.f);
          pe[q] = q < ne ? a.S[first + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        bt[0] = v3.x; bt[1] = v3.y; bt[2] = v3.z;
        const f3 climit = xyz(v2);
        key = __float_as_uint(v2.w);
        if (!chk(key < (uint32_t)c.n_cells, MARS_CHECK_CELL, ctr)) key = 0xffffffffu;
        if (gN > 0) {
          f3 sum = mk3(0.f, 0.f, 0.f);
          for (int k = 0; k < gN; k += 4) {
            if (k > 0) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                pn[q] = k + q < gN ? a.SH[2][sf + k + q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (k + q >= gN) break;
              const f3 v = xyz(pn[q]);
              sum = sum + v;
              const f3 vc = fmin3(v, climit);
              st[1][1] += vc.x; st[1][2] += vc.y; st[1][3] += vc.z;
              st[1][4] += vc.x * vc.x; st[1][5] += vc.y * vc.y; st[1][6] += vc.z * vc.z;
            }
          }
          const float ib1 = 1.0f / bt[1];
          Lr = mk3(sum.x * ib1, sum.y * ib1, sum.z * ib1);
          csub += (uint32_t)gN;
          st[1][0] = (float)gN;
          st[1][7] = (float)gN;
        }
        // 1 / beta once per technique, not one division per child value
        const float ib0 = gB > 0 ? 1.0f / bt[0] : 0.0f, ib2 = gG > 0 ? 1.0f / bt[2] : 0.0f;
        for (int k = 0; k < ne; k += 4) {
          if (k > 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) pe[q] = k + q < ne ? a.S[first + k + q] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (k + q >= ne) break;
            const float4 sv = pe[q];
            const int t = k + q < gB ? 0 : 2;
            const float ib = t == 0 ? ib0 : ib2;
            Lr = Lr + mk3(sv.x * ib, sv.y * ib, sv.z * ib);
            const uint32_t cc = __float_as_uint(sv.w);
            csub += cc;
            const f3 vc = fmin3(xyz(sv), climit);
            if (t == 0) {
              st[0][0] += 1.0f; st[0][1] += vc.x; st[0][2] += vc.y; st[0][3] += vc.z;
              st[0][4] += vc.x * vc.x; st[0][5] += vc.y * vc.y; st[0][6] += vc.z * vc.z; st[0][7] += (float)cc;
            } else {
              st[2][0] += 1.0f; st[2][1] += vc.x; st[2][2] += vc.y; st[2][3] += vc.z;
              st[2][4] += vc.x * vc.x; st[2][5] += vc.y * vc.y; st[2][6] += vc.z * vc.z; st[2][7] += (float)cc;
            }
          }
        }
        if (BD && gL > 0) {
          // light connection samples: the sum of the sample's connections (in
          // the order of its light vertices) and its cost from the light kernels
          unsigned long long lf = __float_as_uint(v3.w);
          if (!chk(lf + (unsigned long long)gL <= a.lcap, MARS_CHECK_ARENA, ctr)) gL = 0;
          const float ib = 1.0f / bt[2];
          for (int q = 0; q < gL; ++q) {
            const float4 lr = a.LR[lf + q];
            const unsigned long long vf = __float_as_uint(lr.x);
            int m = (int)__float_as_uint(lr.y);
            if (!chk(m <= LIGHT_MAX && vf + (unsigned long long)m <= a.vcap, MARS_CHECK_ARENA, ctr)) m = 0;
            f3 v = mk3(0.f, 0.f, 0.f);
            for (int k = 0; k < m; ++k) v = v + xyz(a.LC[vf + k]);
            const uint32_t cc = (uint32_t)lr.w;
            Lr = Lr + mk3(v.x * ib, v.y * ib, v.z * ib);
            csub += cc;
            st[2][0] += 1.0f; st[2][1] += v.x; st[2][2] += v.y; st[2][3] += v.z;
            st[2][4] += v.x * v.x; st[2][5] += v.y * v.y; st[2][6] += v.z * v.z; st[2][7] += (float)cc;
          }
        }
        const f3 G = xyz(v1);
        E = E + mul(G, Lr);
      }
      const uint32_t cost = 1u + csub;
      a.S[i] = f4(E, __uint_as_float(cost));
      if (d == 1 && chk(it.tile_begin + li < (unsigned long long)c.n_pixels, MARS_CHECK_PIXEL, ctr))
        c.img[it.tile_begin + li] = f4(E, (float)cost);  // w: rays of the pixel's path tree
      if (guide_dep) {
        const float wdep = (v4.x + lum(Lr)) * v4.y;
        if (wdep > 0.0f && chk(__float_as_uint(v4.z) < (uint32_t)c.n_cells, MARS_CHECK_CELL, ctr) &&
            chk(__float_as_int(v4.w) >= 0 && __float_as_int(v4.w) < GUIDE_BINS, MARS_CHECK_BIN, ctr)) {
          const uint32_t pc = __float_as_uint(v4.z);
          atomicAdd(c.guide_hist + (size_t)pc * GUIDE_BINS + __float_as_int(v4.w), wdep);
          c.guide_dirty[pc] = 1;
        }
      }
    }

    // ---- iteration counters, kept per thread over all chunks of the launch
    if (active && (flags & F_TRACED)) ++n_traced;
    if (active && (flags & F_EST)) {
      ++n_est;
      sb0 += bt[0];
      sb1 += bt[1];
      sb2 += bt[2];
    }
    if (active && d == 1) n_rays += 1ull + csub;

    // ---- local statistics: reduce runs of equal cells, then float64 atomics
    if (collect) {
      const unsigned any = __ballot_sync(FULL, key != 0xffffffffu);
      if (any) {
        const uint32_t prev = __shfl_up_sync(FULL, key, 1);
        const bool head = lane == 0 || prev != key;
        const unsigned heads = __ballot_sync(FULL, head);
        // a run of two or more lanes with statistics is the only case that needs
        // the segmented scan (in deep waves neighbouring vertices rarely share a cell)
        const bool pairs = __any_sync(FULL, !head && key != 0xffffffffu);
        const unsigned below = lane == 31 ? FULL : ((2u << lane) - 1u);
        const int start = 31 - __clz(heads & below);
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          if (!slot_on(c.techniques, t)) continue;
          // skip a technique no lane drew, and the scan when every run is one lane
          if (!__any_sync(FULL, st[t][0] > 0.0f)) continue;
          if (pairs) {
#pragma unroll
            for (int k = 0; k < NSTAT; ++k) st[t][k] = seg_scan(st[t][k], lane, start);
          }
          if (tail && key != 0xffffffffu && st[t][0] > 0.0f) {
            if (c.stats32) {
              float4* dst = reinterpret_cast<float4*>(c.stats32 + ((size_t)key * NT + t) * NSTAT);
              atomicAdd(dst, make_float4(st[t][0], st[t][1], st[t][2], st[t][3]));
              atomicAdd(dst + 1, make_float4(st[t][4], st[t][5], st[t][6], st[t][7]));
            } else {
              // structure of arrays: the 8 sums of a record sit in 8 different
              // cache lines, so their atomics do not queue on one line
              const size_t plane = (size_t)c.n_cells * NT;
              double* dst = c.stats + (size_t)key * NT + t;
#pragma unroll
              for (int k = 0; k < NSTAT; ++k) atomicAdd(dst + k * plane, (double)st[t][k]);
            }
          }
        }
      }
    }
  }

  // ---- flush the iteration counters: one atomic per counter and warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n_traced += __shfl_xor_sync(FULL, n_traced, off);
    n_est += __shfl_xor_sync(FULL, n_est, off);
    n_rays += __shfl_xor_sync(FULL, n_rays, off);
    sb0 += __shfl_xor_sync(FULL, sb0, off);
    sb1 += __shfl_xor_sync(FULL, sb1, off);
    sb2 += __shfl_xor_sync(FULL, sb2, off);
  }
  if (lane == 0) {
    if (n_traced) atomicAdd(&ctr->vertices, n_traced);
    if (n_est) {
      atomicAdd(&ctr->est_vertices, n_est);
      atomicAdd(&ctr->sum_beta[0], sb0);
      if (on_n) atomicAdd(&ctr->sum_beta[1], sb1);
      if (on_g || BD) atomicAdd(&ctr->sum_beta[2], sb2);
    }
    if (n_rays) atomicAdd(&ctr->rays, n_rays);
  }
}

size_t shade_smem(int threads) { return (size_t)(threads / 32) * sizeof(ShadeWarpCtx); }

// Register-cap variants of every wave kernel: variant v is compiled with
// __launch_bounds__(256, MINB) for MINB = 1 (the compiler's choice), or a cap
// that lets more blocks share an SM (shade and reverse: 80 and 64 registers;
// trace and shadow: 64 and 40 registers), trading spills for occupancy.
using TraceFn = void (*)(const DevScene, const DevCache, const Arena, const IterArgs*, const int);
using ShadowFn = void (*)(const DevScene, const DevCache, const Arena, const int);
TraceFn trace_fn(int v) { return v == 2 ? k_trace<6> : (v == 1 ? k_trace<4> : k_trace<1>); }
TraceFn shade_fn(int v, bool bd = false) {
  if (bd) return v == 2 ? k_shade<4, true> : (v == 1 ? k_shade<3, true> : k_shade<1, true>);
  return v == 2 ? k_shade<4, false> : (v == 1 ? k_shade<3, false> : k_shade<1, false>);
}
ShadowFn shadow_fn(int v) { return v == 2 ? k_shadow<6> : (v == 1 ? k_shadow<4> : k_shadow<1>); }
TraceFn reverse_fn(int v, bool bd = false) {
  if (bd) return v == 2 ? k_reverse<4, true> : (v == 1 ? k_reverse<3, true> : k_reverse<1, true>);
  return v == 2 ? k_reverse<4, false> : (v == 1 ? k_reverse<3, false> : k_reverse<1, false>);
}

}  // namespace

int wave_variants(int) { return 3; }
int wave_variant_registers(int kernel, int v) {
  if (v == 0) return 0;
  if (kernel == WK_SHADE || kernel == WK_REVERSE) return v == 1 ? 80 : 64;
  return v == 1 ? 64 : 40;
}

cudaError_t wave_occupancy(const int threads[WAVE_KERNELS], const int variant[WAVE_KERNELS],
                           int blocks_per_sm[WAVE_KERNELS]) {
  cudaError_t e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[WK_TRACE], trace_fn(variant[WK_TRACE]),
                                                         threads[WK_TRACE], 0)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[WK_SHADE], shade_fn(variant[WK_SHADE]),
                                                         threads[WK_SHADE], shade_smem(threads[WK_SHADE]))) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[WK_SHADOW], shadow_fn(variant[WK_SHADOW]),
                                                         threads[WK_SHADOW], 0)) != cudaSuccess)
    return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[WK_REVERSE], reverse_fn(variant[WK_REVERSE]),
                                                       threads[WK_REVERSE], 0);
}

bool wave_threads_ok(int threads) { return threads >= 32 && threads <= MAX_WAVE_THREADS && threads % 32 == 0; }

cudaError_t launch_tile(const DevScene& s, const DevCache& c, const Arena& a, const IterArgs* it, const WaveLaunch& L,
                        cudaStream_t st, cudaStream_t side, cudaStream_t side2, const cudaEvent_t* sync,
                        cudaEvent_t* ev) {
  k_tile_init<<<1, 32, 0, st>>>(c.ctr, it);
  const int D = c.max_depth;
  const int tT = L.threads[WK_TRACE], tS = L.threads[WK_SHADE], tH = L.threads[WK_SHADOW], tR = L.threads[WK_REVERSE];
  auto G = [&](int k, int) { return L.grid[k]; };
  const size_t smS = shade_smem(tS);
  const bool nee = (c.techniques & MARS_TECH_NEE) != 0;
  const bool bd = (c.techniques & MARS_TECH_LIGHT) != 0;
  // The NEE shadow rays of wave d run on the side stream and its light
  // connection samples on a second one (side2, else the side stream too),
  // overlapped with the forward kernels of the next waves and with each other
  // (disjoint data); the reverse pass, their only consumer, waits for all of
  // them.
  // sync: D + 2 events without timing (after shade(d); after the last shadow
  // kernel; after the last light kernel).  ev (optional, 7 D + 2 timing
  // events): ev[0] start; ev[2(d-1)+1],
  // ev[2(d-1)+2] after wave d's trace and shade; ev[2D + 2(d-1) + 1 .. 2] around
  // its shadow kernel on the side stream; ev[5D + 1] when the reverse pass may
  // start; ev[4D + k] after the k-th reverse kernel; ev[5D + 2 + 2(d-1) .. + 1]
  // around its light connection kernel on the side stream.
  if (ev) cudaEventRecord(ev[0], st);
  cudaStream_t lside = side2 ? side2 : side;
  bool any_shadow = false, any_light = false;
  for (int d = 1; d <= D; ++d) {
    trace_fn(L.variant[WK_TRACE])<<<G(WK_TRACE, d), tT, 0, st>>>(s, c, a, it, d);
    if (ev) cudaEventRecord(ev[2 * (d - 1) + 1], st);
    shade_fn(L.variant[WK_SHADE], bd)<<<G(WK_SHADE, d), tS, smS, st>>>(s, c, a, it, d);
    if (ev) cudaEventRecord(ev[2 * (d - 1) + 2], st);
    const bool shadow = d <= D - 1 && nee, light = bd && d <= D - 2;
    if (shadow || light) cudaEventRecord(sync[d - 1], st);
    if (shadow) {
      cudaStreamWaitEvent(side, sync[d - 1], 0);
      any_shadow = true;
      if (ev) cudaEventRecord(ev[2 * D + 2 * (d - 1) + 1], side);
      shadow_fn(L.variant[WK_SHADOW])<<<G(WK_SHADOW, d), tH, 0, side>>>(s, c, a, d);
      if (ev) cudaEventRecord(ev[2 * D + 2 * (d - 1) + 2], side);
    }
    if (light) {
      if (lside != side || !shadow) cudaStreamWaitEvent(lside, sync[d - 1], 0);
      any_light = true;
      if (ev) cudaEventRecord(ev[5 * D + 2 + 2 * (d - 1)], lside);
      cudaError_t e = launch_light(s, c, a, it, L.variant[WK_SHADOW], G(WK_SHADOW, d), tH, d, lside);
      if (e != cudaSuccess) return e;
      if (ev) cudaEventRecord(ev[5 * D + 2 + 2 * (d - 1) + 1], lside);
    }
  }
  if (any_shadow) {
    cudaEventRecord(sync[D], side);
    cudaStreamWaitEvent(st, sync[D], 0);
  }
  if (any_light && lside != side) {
    cudaEventRecord(sync[D + 1], lside);
    cudaStreamWaitEvent(st, sync[D + 1], 0);
  } else if (any_light && !any_shadow) {
    cudaEventRecord(sync[D], side);
    cudaStreamWaitEvent(st, sync[D], 0);
  }
  if (ev) cudaEventRecord(ev[5 * D + 1], st);
  for (int d = D; d >= 1; --d) {
    reverse_fn(L.variant[WK_REVERSE], bd)<<<G(WK_REVERSE, d), tR, 0, st>>>(s, c, a, it, d);
    if (ev) cudaEventRecord(ev[4 * D + (D - d + 1)], st);
  }
  k_tile_finish<<<1, 32, 0, st>>>(c.ctr, c.tile_status, it, D);
  return cudaGetLastError();
}

cudaError_t launch_merge_lanes(DevCounters* dst, DevCounters* src, cudaStream_t st) {
  k_merge_lanes<<<1, 32, 0, st>>>(dst, src);
  return cudaGetLastError();
}

int tile_launches(int max_depth, int techniques) {
  // light connections: a light-subpath and a connection kernel per wave of depth <= D - 2
  return 2 + 2 * max_depth + max_depth + ((techniques & MARS_TECH_NEE) ? max_depth - 1 : 0) +
         ((techniques & MARS_TECH_LIGHT) && max_depth > 2 ? 2 * (max_depth - 2) : 0);
}

}  // namespace mars
