// bdpt.cu -- the light connection technique of the bidirectional application
// (Sec. 5): per light connection sample drawn at camera vertex x_i (by the
// shade kernel of wave i), one light subpath and its weighted connections to
// x_i, in two kernels per wave:
//
//   k_light_path (wave i)     one thread per sample: the light subpath (a light
//                             chosen as for NEE, a uniform point y_0, cosine
//                             emission, at every surface vertex y_k BSDF
//                             sampling with the light arriving from y_{k-1} and
//                             throughput-based Russian roulette -- survival
//                             q = min(1, max_ch f cos / p), the throughput
//                             divided by it; Sec. 5 never splits light paths --
//                             up to LIGHT_MAX and D - 1 - i surface vertices),
//                             its vertices written to the light vertex region
//                             with what the weights need of each; the sample's
//                             cost is the rays of its subpath plus one per
//                             connection.
//   k_light_connect (wave i)  one thread per light vertex y_k: the connection
//                             x_i -- y_k, its contribution alpha_k f_y f_x / d^2,
//                             its balance weight over every strategy of the
//                             full path, and a shadow ray.
//
// The sample's value, the sum of its visible weighted connections in the order
// of its light vertices, is formed by the reverse pass.
//
// The weight of connection x_i -- y_j relative to the camera prefix C_i:
//   (a) this strategy:            bw_L(x_i) lambda_j  (lambda_j: area density of
//                                  y_j on the light subpath, pN included)
//   (b) connections before x_i:   lambda_j P<-_i sum_{l <= LIGHT_MAX - j} W_i[l]
//       (W_i[1] = Y_i[1], W_i[l] = Y_i[l] P<-_{i-1}; see render.cu)
//   (c) strategies that reach y_j..y_1 as camera vertices: the camera prefix
//       continued through them (bw_B P-> per step, with each vertex's budgets
//       from the count rule at its cell with the throughput of a camera path
//       through it), adding there a light connection to the rest of the
//       subpath (bw_L lambda), NEE at y_1 (bw_N pN) and the camera path that
//       hits y_0.
#include "device.cuh"

namespace mars {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_LIGHT_THREADS = 256;

struct LightVertex {
  f3 p, l, alpha;  // position, unit direction towards the previous light vertex, throughput
  f3 ng;           // geometric normal
  float t, lam;    // distance to the previous light vertex, area density on the subpath
  int prim;
  Mat mat;
};

__device__ __forceinline__ Mat material_at(const DevScene& s, int prim, DevCounters* ctr, float4* m0_out) {
  int m = prim_material(s.prims, prim);
  if (!chk(m >= 0 && m < s.n_mats, MARS_CHECK_MATERIAL, ctr)) m = 0;
  const float4 m0 = __ldg(s.mats + 3 * m), m1 = __ldg(s.mats + 3 * m + 1);
  Mat mt;
  mt.type = (int)m0.x;
  mt.alpha = m0.y;
  mt.col = xyz(m1);
  if (m0_out) *m0_out = m0;
  return mt;
}

__device__ __forceinline__ float4 f4(f3 a, float w) { return make_float4(a.x, a.y, a.z, w); }

// inclusive prefix sum of n over the warp's lanes (x) and the warp's total (y)
__device__ __forceinline__ int2 warp_scan_incl(int n, int lane) {
  int v = n;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int u = __shfl_up_sync(FULL, v, off);
    if (lane >= off) v += u;
  }
  return make_int2(v, __shfl_sync(FULL, v, 31));
}

// first light vertex slot of wave d: the earlier waves' vertices come first
// (their light kernels ran before on the same stream)
__device__ __forceinline__ unsigned long long vertex_base(const DevCounters* ctr, int d) {
  unsigned long long b = 0;
  for (int e = 1; e < d; ++e) b += ctr->vcount[e];
  return b;
}

// One thread per light connection sample of wave d (a warp-uniform loop: the
// light vertex slots are allocated per warp): its light subpath, then the
// per-vertex terms the connections' weights need, written to the light vertex
// region; LR = (first vertex slot, m, pN, cost).
template <int MINB>
__global__ void __launch_bounds__(MAX_LIGHT_THREADS, MINB) k_light_path(const DevScene s, const DevCache c,
                                                               const Arena a, const IterArgs* __restrict__ itp,
                                                               const int d) {
  const IterArgs it = *itp;
  DevCounters* ctr = c.ctr;
  if (ctr->overflow) return;  // the tile is re-rendered
  const unsigned long long lb = ctr->lbase[d], lc = ctr->lcount[d];
  const unsigned long long n = lb >= a.lcap ? 0ull : (lc < a.lcap - lb ? lc : a.lcap - lb);
  const unsigned long long vb = vertex_base(ctr, d);
  const Rng rng{it.seed, it.job, it.iteration};
  const int D = c.max_depth;
  const int lane = threadIdx.x & 31;
  TraceWork tw;
  unsigned long long n_rays = 0;
  const unsigned long long w0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull;
  for (unsigned long long b0 = w0; b0 < n; b0 += gridDim.x * (unsigned long long)blockDim.x) {
    const unsigned long long k = b0 + lane;
    const bool active = k < n;
    const unsigned long long j = lb + k;
    LightVertex y[LIGHT_MAX];
    int m = 0, rays = 0;
    float pN = 0.0f, cos0 = 0.0f;
    if (active) {
      const float4 j0 = a.LJ[0][j], j1 = a.LJ[1][j], j7 = a.LJ[7][j];
      uint32_t px = __float_as_uint(j0.w);
      if (!chk(px < (uint32_t)c.n_pixels, MARS_CHECK_PIXEL, ctr)) px = 0;
      const uint32_t bits = __float_as_uint(j1.w);
      const int sidx = (int)((bits >> 8) & 0xffu), depth_i = (int)(bits >> 16);
      const uint64_t lin = (uint64_t)__float_as_uint(j7.x) | ((uint64_t)__float_as_uint(j7.y) << 32);
      int kmax = D - 1 - depth_i;
      if (kmax > LIGHT_MAX) kmax = LIGHT_MAX;

      // ---- y_0 on a light (chosen by area x radiance, as NEE)
      float4 u = rng.u4(px, DIM_LIGHT + 8u * (uint32_t)sidx, lin);
      int l = s.n_lights - 1;
      for (int q = 0; q < s.n_lights; ++q)
        if (u.x < __ldg(&s.lights[5 * q].w)) { l = q; break; }
      const float4 l0 = __ldg(s.lights + 5 * l), l1 = __ldg(s.lights + 5 * l + 1), l2 = __ldg(s.lights + 5 * l + 2),
                   l3 = __ldg(s.lights + 5 * l + 3), l4 = __ldg(s.lights + 5 * l + 4);
      const f3 y0 = xyz(l0) + (xyz(l1) * u.y + xyz(l2) * u.z);
      const f3 nl = xyz(l3);
      pN = l1.w / l2.w;
      // cosine-distributed emission direction about the light's normal
      u = rng.u4(px, DIM_LIGHT + 8u * (uint32_t)sidx + 1u, lin);
      const Frame fl = make_frame(nl);
      float sp, cp;
      sincospif(2.0f * u.y, &sp, &cp);   // sin, cos of 2 pi u.y (2 u.y is exact)
      const float r = sqrtf(u.x), zc = 1.0f - u.x;
      const f3 dir0 = fl.to_world(mk3(r * cp, r * sp, sqrtf(zc > 0.0f ? zc : 0.0f)));
      cos0 = dot(nl, dir0);
      // alpha_1 = Le cos / (pN cos / pi) = Le pi / pN
      f3 alpha = xyz(l4) * (PI_F / pN);
      f3 org = y0 + nl * s.eps, dir = dir0;
      float pdens = cos0 * INV_PI_F;   // solid-angle density of the next vertex's direction
      // the loops stay rolled: unrolled, the compiler keeps every vertex of y in
      // registers (235 per thread, 8 warps per SM); rolled, y lives in the
      // thread's local frame (L1) and the kernel takes 112 (config 3 at 1024^2:
      // light kernels 3.27 -> 2.74 ms alone, iteration 7.7 -> 6.7 ms)
#pragma unroll 1
      for (int kk = 1; kk <= kmax; ++kk) {
        ++rays;
        float t = 0.0f;
        const int prim = trace_closest(s, org, dir, t, tw);
        if (prim < 0 || !chk(prim < s.n_prims, MARS_CHECK_PRIM, ctr)) break;
        const f3 p = org + dir * t;
        const f3 ng = prim_normal(s.prims, prim, p);
        float4 m0;
        const Mat mt = material_at(s, prim, ctr, &m0);
        if (!(m0.z > 0.0f)) break;   // a surface that reflects nothing ends the subpath
        const float lam = (kk == 1 ? pN : y[kk - 2].lam) * pdens * fabsf(dot(ng, dir)) / (t * t);
        const f3 lin_dir = dir * -1.0f;
        y[kk - 1].p = p;
        y[kk - 1].l = lin_dir;
        y[kk - 1].alpha = alpha;
        y[kk - 1].ng = ng;
        y[kk - 1].t = t;
        y[kk - 1].lam = lam;
        y[kk - 1].prim = prim;
        y[kk - 1].mat = mt;
        m = kk;
        if (kk == kmax) break;
        // continue: BSDF sampling with the light arriving from y_{k-1}, then the roulette
        u = rng.u4(px, DIM_LIGHT + 8u * (uint32_t)sidx + (uint32_t)kk + 1u, lin);
        const f3 ns = dot(ng, lin_dir) >= 0.0f ? ng : ng * -1.0f;
        const Frame fr = make_frame(ns);
        const f3 lloc = fr.to_local(lin_dir);
        f3 wl;
        if (!bsdf_sample(mt, lloc, u.x, u.y, wl)) break;
        float pB;
        const f3 fc = bsdf_eval(mt, lloc, wl, pB);
        if (!(pB > 0.0f) || !nonzero(fc)) break;
        const float q = fminf(1.0f, max_channel(fc) / pB);
        if (!(u.z < q)) break;   // Russian roulette, decided in float32
        const float iq = 1.0f / (pB * q);
        alpha = mul(alpha, fc) * iq;
        org = p + ns * s.eps;
        dir = fr.to_world(wl);
        pdens = pB * q;
      }
      n_rays += (unsigned long long)rays;
    }

    // ---- m light vertex slots per sample: one atomic per warp
    const int2 sc = warp_scan_incl(m, lane);
    unsigned long long wb = 0;
    if (lane == 31 && sc.y > 0) wb = atomicAdd(&ctr->vcount[d], (unsigned long long)sc.y);
    wb = __shfl_sync(FULL, wb, 31);
    const unsigned long long vfirst = vb + wb + (unsigned long long)(sc.x - m);
    if (active) {
      if (m > 0 && vfirst + (unsigned long long)m > a.vcap) {
        atomicOr(&ctr->overflow, 1u);
        m = 0;
      }
      // what the connections' weights need of each light vertex: its cell, the
      // reverse BSDF towards the previous vertex with the next one as the
      // outgoing direction (the last vertex's depends on the connection), and
      // the cosine at the previous vertex towards it
#pragma unroll 1
      for (int kk = 1; kk <= m; ++kk) {
        const LightVertex& v = y[kk - 1];
        int cell = c.oct_nodes ? octree_cell(s, c.oct_nodes, v.p) : cell_of(s, c.grid_n, v.p);
        if (!chk(cell >= 0 && cell < c.n_cells, MARS_CHECK_CELL, ctr)) cell = 0;
        const float cos_prev = kk == 1 ? cos0 : fabsf(dot(y[kk - 2].ng, v.l));
        f3 frev = mk3(0.f, 0.f, 0.f);
        float prev = 0.0f;
        if (kk < m) {
          const f3 wo_u = y[kk].l * -1.0f;
          const f3 nsu = dot(v.ng, wo_u) >= 0.0f ? v.ng : v.ng * -1.0f;
          const Frame fu = make_frame(nsu);
          frev = bsdf_eval(v.mat, fu.to_local(wo_u), fu.to_local(v.l), prev);
        }
        const unsigned long long vs = vfirst + (unsigned long long)(kk - 1);
        a.LV[0][vs] = f4(v.p, __int_as_float(v.prim));
        a.LV[1][vs] = f4(v.l, v.t);
        a.LV[2][vs] = f4(v.alpha, v.lam);
        a.LV[3][vs] = f4(v.ng, __int_as_float(cell));
        a.LV[4][vs] = f4(frev, prev);
        a.LV[5][vs] = make_float4(cos_prev, __uint_as_float((uint32_t)k), __int_as_float(kk - 1), 0.0f);
      }
      a.LR[j] = make_float4(__uint_as_float((uint32_t)vfirst), __uint_as_float((uint32_t)m), pN, (float)(rays + m));
    }
  }
#ifdef MARS_CHECKED
  if (tw.bad) atomicOr(&ctr->check_flags, tw.bad);
#endif
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) n_rays += __shfl_xor_sync(FULL, n_rays, off);
  if (lane == 0 && n_rays) atomicAdd(&ctr->light_rays, n_rays);
}

// One thread per light vertex y_k of wave d's samples: the connection x_i --
// y_k, its contribution alpha_k f_y f_x / d^2, its balance weight over every
// strategy of the full path, and a shadow ray; LC = the weighted contribution
// if visible, else zero.
template <int MINB>
__global__ void __launch_bounds__(MAX_LIGHT_THREADS, MINB) k_light_connect(const DevScene s, const DevCache c,
                                                                  const Arena a, const IterArgs* __restrict__ itp,
                                                                  const int d) {
  const IterArgs it = *itp;
  DevCounters* ctr = c.ctr;
  if (ctr->overflow) return;  // the tile is re-rendered
  const unsigned long long lb = ctr->lbase[d];
  const unsigned long long vb = vertex_base(ctr, d), vc = ctr->vcount[d];
  const unsigned long long n = vb >= a.vcap ? 0ull : (vc < a.vcap - vb ? vc : a.vcap - vb);
  const int D = c.max_depth;
  const bool on_n = c.techniques & MARS_TECH_NEE;
  const bool aware = it.aware != 0;
  TraceWork tw;
  unsigned long long n_conn = 0;
  for (unsigned long long q0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q0 < n;
       q0 += gridDim.x * (unsigned long long)blockDim.x) {
    const unsigned long long vs = vb + q0;
    const float4 v5 = a.LV[5][vs];
    const unsigned long long ks = __float_as_uint(v5.y);
    const int kk = __float_as_int(v5.z) + 1;   // 1-based index on the subpath
    if (!chk(ks < a.lcap - lb && kk >= 1 && kk <= LIGHT_MAX && vs + 1 >= (unsigned long long)kk, MARS_CHECK_ARENA,
             ctr)) {
      a.LC[vs] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const unsigned long long j = lb + ks;
    const unsigned long long vfirst = vs + 1 - (unsigned long long)kk;
    const float4 j0 = a.LJ[0][j], j1 = a.LJ[1][j], j2 = a.LJ[2][j], j3 = a.LJ[3][j], j4 = a.LJ[4][j],
                 j5 = a.LJ[5][j], j6 = a.LJ[6][j];
    const float pN = a.LR[j].z;
    const f3 xo = xyz(j0);
    uint32_t px = __float_as_uint(j0.w);
    if (!chk(px < (uint32_t)c.n_pixels, MARS_CHECK_PIXEL, ctr)) px = 0;
    const f3 nsx = xyz(j1);
    const uint32_t bits = __float_as_uint(j1.w);
    Mat mx;
    mx.type = (int)(bits & 0xffu);
    mx.alpha = j2.w;
    mx.col = xyz(j2);
    const int depth_i = (int)(bits >> 16);
    const f3 wo_x = xyz(j3), T_x = xyz(j4);
    const float mult_x = j3.w, betaB_x = j4.w;
    const float bwB_x = j5.x, bwL_x = j5.z, gprev = j5.w;
    const float Y[4] = {j6.x, j6.y, j6.z, j6.w};

    // the connected vertex y_kk
    const float4 v0 = a.LV[0][vs], v1 = a.LV[1][vs], v2 = a.LV[2][vs], v3 = a.LV[3][vs];
    const f3 yp = xyz(v0), yl = xyz(v1), yalpha = xyz(v2), ngk = xyz(v3);
    const float ylam = v2.w;
    int yprim = __float_as_int(v0.w);
    if (!chk(yprim >= 0 && yprim < s.n_prims, MARS_CHECK_PRIM, ctr)) yprim = 0;
    const Frame fx = make_frame(nsx);
    const f3 wox = fx.to_local(wo_x);
    const f3 nsy = dot(ngk, yl) >= 0.0f ? ngk : ngk * -1.0f;
    const f3 yo = yp + nsy * s.eps;
    const f3 dv = yo - xo;
    const float d2 = dot(dv, dv);
    const float dist = sqrtf(d2);
    const f3 w = dv * (1.0f / dist);
    const f3 wx = fx.to_local(w);
    float pxv;
    const f3 fxv = bsdf_eval(mx, wox, wx, pxv);
    const Mat my = material_at(s, yprim, ctr, nullptr);
    const Frame fy = make_frame(nsy);
    const f3 ly = fy.to_local(yl), wy = fy.to_local(w * -1.0f);
    float pyv;
    const f3 fyv = bsdf_eval(my, ly, wy, pyv);
    const float id2 = 1.0f / d2;
    const f3 C = mul(mul(yalpha, fyv), fxv) * id2;
    f3 val = mk3(0.f, 0.f, 0.f);
    if (nonzero(C)) {
      // (a) this strategy
      const float ta = bwL_x * ylam;
      // (b) light connections at camera vertices before x_i
      // (terms l = 1 .. LIGHT_MAX - kk back: W[1] = Y[1], W[l] = Y[l] P<-_{i-1})
      float tb = 0.0f;
      const float y1 = LIGHT_MAX - kk >= 1 ? Y[0] : 0.0f;
      float sw = 0.0f;
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (q < LIGHT_MAX - kk) sw += Y[q];
      if (y1 > 0.0f || sw > 0.0f) {
        const float qy = pyv > 0.0f ? fminf(1.0f, max_channel(fyv) / pyv) : 0.0f;
        const float lpi = pyv * qy * fabsf(dot(nsx, w)) * id2;
        float lp = 0.0f;
        if (sw > 0.0f) {
          float prev;
          const f3 frev = bsdf_eval(mx, wx, wox, prev);
          const float qx = prev > 0.0f ? fminf(1.0f, max_channel(frev) / prev) : 0.0f;
          lp = prev * qx * gprev;
        }
        tb = ylam * lpi * (y1 + lp * sw);
      }
      // (c) the strategies that reach y_kk..y_1 as camera vertices
      float G = bwB_x * pxv * fabsf(dot(ngk, w)) * id2;
      f3 Tu = pxv > 0.0f ? mul(T_x, fxv) * (1.0f / (pxv * betaB_x)) : mk3(0.f, 0.f, 0.f);
      float mu = mult_x * betaB_x;
      float tc = 0.0f;
      f3 wo_u = w * -1.0f;   // towards the camera side
      const float4 est = it.has_estimate ? c.est[px] : make_float4(1.f, 1.f, 1.f, 0.f);
      for (int a_ = 1; a_ <= kk; ++a_) {
        const unsigned long long us = vfirst + (unsigned long long)(kk - a_);   // y_{kk - a_ + 1}
        const float4 u1 = a.LV[1][us], u3 = a.LV[3][us], u5 = a.LV[5][us];
        const f3 ul = xyz(u1);
        int ucell = __float_as_int(u3.w);
        if (!chk(ucell >= 0 && ucell < c.n_cells, MARS_CHECK_CELL, ctr)) ucell = 0;
        const int depth_u = depth_i + a_;
        const bool lc_here = depth_u <= D - 2;
        const unsigned on_mask = 1u | (on_n ? 2u : 0u) | (lc_here ? 4u : 0u);
        float bu[NT];
        vertex_budgets(c, it, ucell, Tu, est, mu, on_mask, 1.0f, 1.0f, bu);
        const float bwBu = aware ? bu[0] : 1.0f;
        const float bwNu = on_n ? (aware ? bu[1] : 1.0f) : 0.0f;
        const float bwLu = lc_here ? (aware ? bu[2] : 1.0f) : 0.0f;
        float pBu;
        f3 fcu;
        if (a_ == 1) {
          // the connected vertex: the camera side arrives along the connection
          const f3 ung = xyz(u3);
          const f3 nsu = dot(ung, wo_u) >= 0.0f ? ung : ung * -1.0f;
          const Frame fu = make_frame(nsu);
          fcu = bsdf_eval(my, fu.to_local(wo_u), fu.to_local(ul), pBu);
        } else {
          const float4 u4 = a.LV[4][us];
          fcu = xyz(u4);
          pBu = u4.w;
        }
        if (a_ <= kk - 1) tc += G * bwLu * a.LV[2][us - 1].w;   // lambda of y_{kk - a_}
        if (a_ == kk) tc += G * bwNu * pN;
        G *= bwBu * pBu * u5.x / (u1.w * u1.w);
        Tu = pBu > 0.0f ? mul(Tu, fcu) * (1.0f / (pBu * bu[0])) : mk3(0.f, 0.f, 0.f);
        mu *= bu[0];
        wo_u = ul * -1.0f;
      }
      tc += G;
      const float den = ta + tb + tc;
      const float wgt = den > 0.0f ? ta / den : 0.0f;
      ++n_conn;
      if (!trace_any4(s, xo, w, dist - s.eps, tw)) val = C * wgt;
    }
    a.LC[vs] = f4(val, 0.0f);
  }
#ifdef MARS_CHECKED
  if (tw.bad) atomicOr(&ctr->check_flags, tw.bad);
#endif
  // one atomic per warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) n_conn += __shfl_xor_sync(FULL, n_conn, off);
  if ((threadIdx.x & 31) == 0 && n_conn) atomicAdd(&ctr->conn_rays, n_conn);
}

}  // namespace

int light_variants() { return 3; }

cudaError_t launch_light(const DevScene& s, const DevCache& c, const Arena& a, const IterArgs* it, int variant,
                         int grid, int threads, int d, cudaStream_t st) {
  if (threads > MAX_LIGHT_THREADS) threads = MAX_LIGHT_THREADS;
  if (variant == 2) {
    k_light_path<3><<<grid, threads, 0, st>>>(s, c, a, it, d);
    k_light_connect<3><<<grid, threads, 0, st>>>(s, c, a, it, d);
  } else if (variant == 1) {
    k_light_path<2><<<grid, threads, 0, st>>>(s, c, a, it, d);
    k_light_connect<2><<<grid, threads, 0, st>>>(s, c, a, it, d);
  } else {
    k_light_path<1><<<grid, threads, 0, st>>>(s, c, a, it, d);
    k_light_connect<1><<<grid, threads, 0, st>>>(s, c, a, it, d);
  }
  return cudaGetLastError();
}

}  // namespace mars
