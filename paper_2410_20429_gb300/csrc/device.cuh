// device.cuh -- device-side building blocks of the MARS wavefront kernels:
// counter-based RNG, vector math, ray/primitive intersection, BVH traversal,
// BSDFs and the guided technique's directional histogram.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace mars {

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., "Parallel Random Numbers: As Easy as 1, 2, 3",
// SC 2011): ten rounds, each two 32x32 -> 64-bit products of counter words 0
// and 2 with 0xD2511F53 / 0xCD9E8D57, the high halves xor-ed with the other
// two words and the round key; the key advances by (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Counter layout: (pixel, iteration << 16 | dimension, lineage lo, lineage hi),
// key (seed, job).  Uniforms keep the top 24 bits of a word: exact in float.
struct Rng {
  uint32_t seed, job, iter;
  __device__ __forceinline__ float4 u4(uint32_t px, uint32_t dim, uint64_t lin) const {
    uint4 o = philox4x32_10(make_uint4(px, (iter << 16) | dim, (uint32_t)lin, (uint32_t)(lin >> 32)),
                            make_uint2(seed, job));
    const float s = 1.0f / 16777216.0f;
    return make_float4((float)(o.x >> 8) * s, (float)(o.y >> 8) * s, (float)(o.z >> 8) * s,
                       (float)(o.w >> 8) * s);
  }
};

// ------------------------------------------------------------------ vectors
struct f3 {
  float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 xyz(float4 a) { return {a.x, a.y, a.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ f3 mul(f3 a, f3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 normalize(f3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float lum(f3 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }
__device__ __forceinline__ bool nonzero(f3 c) { return c.x > 0.f || c.y > 0.f || c.z > 0.f; }

// ------------------------------------------------------------ intersection
__device__ __forceinline__ bool hit_quad(const float4* q, f3 o, f3 d, float tmax, float& t_out) {
  const f3 p0 = xyz(q[0]), e1 = xyz(q[1]), e2 = xyz(q[2]);
  const f3 n = cross(e1, e2);
  const float den = dot(d, n);
  if (den == 0.0f) return false;
  const float t = dot(p0 - o, n) / den;
  if (!(t > 0.0f && t < tmax)) return false;
  const f3 w = (o + d * t) - p0;
  const float nn = dot(n, n);
  const float a = dot(cross(w, e2), n) / nn;
  const float b = dot(cross(e1, w), n) / nn;
  if (a < 0.0f || a > 1.0f || b < 0.0f || b > 1.0f) return false;
  t_out = t;
  return true;
}

__device__ __forceinline__ bool hit_sphere(const float4* q, f3 o, f3 d, float tmax, float& t_out) {
  const f3 oc = o - xyz(q[0]);
  const float r = q[1].x;
  const float b = dot(oc, d);
  // b^2 - (|oc|^2 - r^2) = r^2 - |oc - b d|^2 for a unit d; the second form
  // keeps float32 precision for rays that pass far from the centre
  const f3 f = oc - d * b;
  const float disc = r * r - dot(f, f);
  if (disc < 0.0f) return false;
  const float sq = sqrtf(disc);
  float t = -b - sq;
  if (!(t > 0.0f)) t = -b + sq;
  if (!(t > 0.0f && t < tmax)) return false;
  t_out = t;
  return true;
}

__device__ __forceinline__ bool hit_tri(const float4* q, f3 o, f3 d, float tmax, float& t_out) {
  const f3 v0 = xyz(q[0]), e1 = xyz(q[1]), e2 = xyz(q[2]);
  const f3 p = cross(d, e2);
  const float det = dot(e1, p);
  if (det == 0.0f) return false;
  const float inv = 1.0f / det;
  const f3 s = o - v0;
  const float a = dot(s, p) * inv;
  if (a < 0.0f || a > 1.0f) return false;
  const f3 qv = cross(s, e1);
  const float b = dot(d, qv) * inv;
  if (b < 0.0f || a + b > 1.0f) return false;
  const float t = dot(e2, qv) * inv;
  if (!(t > 0.0f && t < tmax)) return false;
  t_out = t;
  return true;
}

// Work counters of a traversal (for the arithmetic roofline): node visits
// (two box tests each) and primitive tests by type.
struct TraceWork {
  unsigned int nodes = 0, quads = 0, spheres = 0, tris = 0;
  unsigned int bad = 0;  // checked builds: MARS_CHECK_NODE / MARS_CHECK_PRIM bits of failed checks
};

// checked builds: a node or primitive index the traversal read from the BVH is
// inside the node or primitive array (else the bit is recorded and the
// traversal stops)
__device__ __forceinline__ bool trav_ok(bool ok, unsigned int bit, TraceWork& w) {
#ifdef MARS_CHECKED
  if (!ok) w.bad |= bit;
  return ok;
#else
  (void)bit;
  (void)w;
  return true;
#endif
}

__device__ __forceinline__ bool hit_prim(const float4* __restrict__ prims, int i, f3 o, f3 d, float tmax,
                                         float& t, TraceWork& w) {
  const float4* q = prims + 4 * i;
  const int type = __float_as_int(q[0].w) & 3;
  w.quads += type == PRIM_QUAD;
  w.spheres += type == PRIM_SPHERE;
  w.tris += type == PRIM_TRI;
  if (type == PRIM_QUAD) return hit_quad(q, o, d, tmax, t);
  if (type == PRIM_SPHERE) return hit_sphere(q, o, d, tmax, t);
  return hit_tri(q, o, d, tmax, t);
}

// Three-input minimum and maximum: one instruction on sm_100 and later.  Like
// fminf / fmaxf they return the extreme of the inputs that are not NaN, so a
// chain of them gives the same value as the two-input chain.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// slab test of one box against [0, tmax]; returns the entry distance, or NaN
// on a miss (so that every comparison with it is false)
__device__ __forceinline__ float box_entry(float4 lo, float4 hi, f3 o, f3 inv, float tmax) {
  const float x0 = (lo.x - o.x) * inv.x, x1 = (hi.x - o.x) * inv.x;
  const float y0 = (lo.y - o.y) * inv.y, y1 = (hi.y - o.y) * inv.y;
  const float z0 = (lo.z - o.z) * inv.z, z1 = (hi.z - o.z) * inv.z;
  const float tn = fmax3(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), 0.0f));
  const float tf = fmin3(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), tmax));
  return tn <= tf * 1.00000024f ? tn : __int_as_float(0x7fffffff);
}

constexpr int STACK = 48;

// Closest hit by stack traversal of the LBVH.  Ties in t go to the lower
// primitive index, as in a brute-force scan in index order.
__device__ __forceinline__ int trace_closest(const DevScene& s, f3 o, f3 d, float& t_best, TraceWork& w) {
  t_best = __int_as_float(0x7f800000);
  int best = -1;
  if (s.n_prims == 1) {
    float t;
    if (hit_prim(s.prims, 0, o, d, t_best, t, w)) { t_best = t; best = 0; }
    return best;
  }
  const f3 inv = mk3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int stack[STACK];
  int sp = 0;
  int node = 0;
  // every internal node is visited at most once per ray
  for (int visits = 0; visits < s.n_prims; ++visits) {
    if (!trav_ok(node >= 0 && node < s.n_prims - 1, MARS_CHECK_NODE, w)) break;
    const BvhNode nd = s.nodes[node];
    ++w.nodes;
    // admit boxes entered at t <= t_best (a tie may still win on index)
    const float tl = box_entry(nd.a, nd.b, o, inv, t_best);
    const float tr = box_entry(nd.c, nd.d, o, inv, t_best);
    int cl = __float_as_int(nd.a.w), cr = __float_as_int(nd.b.w);
    bool vl = tl <= t_best, vr = tr <= t_best;
    // the admitted leaf children (left first) go through one copy of the
    // primitive test, so that lanes with a leaf on either side share it
    int p0 = -1, p1 = -1;
    if (vl && cl < 0) {
      p0 = ~cl;
      vl = false;
    }
    if (vr && cr < 0) {
      if (p0 < 0) p0 = ~cr; else p1 = ~cr;
      vr = false;
    }
    while (p0 >= 0) {
      if (!trav_ok(p0 < s.n_prims, MARS_CHECK_PRIM, w)) break;
      float t;
      if (hit_prim(s.prims, p0, o, d, t_best * 1.0000002f + 1e-30f, t, w) &&
          (t < t_best || (t == t_best && p0 < best))) { t_best = t; best = p0; }
      p0 = p1;
      p1 = -1;
    }
    if (vl && vr) {
      const bool lfirst = tl <= tr;
      const int near = lfirst ? cl : cr, far = lfirst ? cr : cl;
      if (sp < STACK) stack[sp++] = far;
      node = near;
    } else if (vl) {
      node = cl;
    } else if (vr) {
      node = cr;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return best;
}

// Entry distances of the four child boxes of a 4-wide node against [0, tmax]
// (NaN for a miss or an empty slot), by the same slab arithmetic as box_entry.
__device__ __forceinline__ void box4_entry(const Bvh4Node& nd, f3 o, f3 inv, float tmax, float t[4]) {
  const float lx[4] = {nd.lox.x, nd.lox.y, nd.lox.z, nd.lox.w}, ly[4] = {nd.loy.x, nd.loy.y, nd.loy.z, nd.loy.w};
  const float lz[4] = {nd.loz.x, nd.loz.y, nd.loz.z, nd.loz.w}, hx[4] = {nd.hix.x, nd.hix.y, nd.hix.z, nd.hix.w};
  const float hy[4] = {nd.hiy.x, nd.hiy.y, nd.hiy.z, nd.hiy.w}, hz[4] = {nd.hiz.x, nd.hiz.y, nd.hiz.z, nd.hiz.w};
  const int ch[4] = {nd.child.x, nd.child.y, nd.child.z, nd.child.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float x0 = (lx[k] - o.x) * inv.x, x1 = (hx[k] - o.x) * inv.x;
    const float y0 = (ly[k] - o.y) * inv.y, y1 = (hy[k] - o.y) * inv.y;
    const float z0 = (lz[k] - o.z) * inv.z, z1 = (hz[k] - o.z) * inv.z;
    const float tn = fmax3(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), 0.0f));
    const float tf = fmin3(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), tmax));
    t[k] = (ch[k] != BVH4_EMPTY && tn <= tf * 1.00000024f) ? tn : __int_as_float(0x7fffffff);
  }
}

// Any hit with 0 < t < tmax over the 4-wide BVH.
__device__ __forceinline__ bool trace_any4(const DevScene& s, f3 o, f3 d, float tmax, TraceWork& w) {
  float th;
  if (s.n_prims == 1) return hit_prim(s.prims, 0, o, d, tmax, th, w);
  const f3 inv = mk3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int stack[STACK];
  int sp = 0;
  int node = 0;
  for (int visits = 0; visits < s.n_nodes4; ++visits) {
    if (!trav_ok(node >= 0 && node < s.n_nodes4, MARS_CHECK_NODE, w)) break;
    const Bvh4Node nd = s.nodes4[node];
    w.nodes += 2;
    float t[4];
    box4_entry(nd, o, inv, tmax, t);
    const int ch[4] = {nd.child.x, nd.child.y, nd.child.z, nd.child.w};
    int next = -1;
    unsigned leaves = 0;  // admitted leaf children, tested below in child order
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!(t[k] <= tmax)) continue;
      if (ch[k] < 0) {
        leaves |= 1u << k;
      } else if (next < 0) {
        next = ch[k];
      } else if (sp < STACK) {
        stack[sp++] = ch[k];
      }
    }
    // one copy of the primitive test for all of them (lanes share it)
    while (leaves) {
      const int k = __ffs(leaves) - 1;
      leaves &= leaves - 1;
      const int c = k == 0 ? ch[0] : (k == 1 ? ch[1] : (k == 2 ? ch[2] : ch[3]));
      if (!trav_ok(~c < s.n_prims, MARS_CHECK_PRIM, w)) return false;
      if (hit_prim(s.prims, ~c, o, d, tmax, th, w)) return true;
    }
    if (next >= 0) {
      node = next;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return false;
}

// Any hit with 0 < t < tmax.
__device__ __forceinline__ bool trace_any(const DevScene& s, f3 o, f3 d, float tmax, TraceWork& w) {
  float t;
  if (s.n_prims == 1) return hit_prim(s.prims, 0, o, d, tmax, t, w);
  const f3 inv = mk3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int stack[STACK];
  int sp = 0;
  int node = 0;
  for (int visits = 0; visits < s.n_prims; ++visits) {
    if (!trav_ok(node >= 0 && node < s.n_prims - 1, MARS_CHECK_NODE, w)) break;
    const BvhNode nd = s.nodes[node];
    ++w.nodes;
    const float tl = box_entry(nd.a, nd.b, o, inv, tmax);
    const float tr = box_entry(nd.c, nd.d, o, inv, tmax);
    const int cl = __float_as_int(nd.a.w), cr = __float_as_int(nd.b.w);
    bool vl = tl <= tmax, vr = tr <= tmax;
    if (vl && cl < 0) {
      if (hit_prim(s.prims, ~cl, o, d, tmax, t, w)) return true;
      vl = false;
    }
    if (vr && cr < 0) {
      if (hit_prim(s.prims, ~cr, o, d, tmax, t, w)) return true;
      vr = false;
    }
    if (vl && vr) {
      if (sp < STACK) stack[sp++] = cr;
      node = cl;
    } else if (vl) {
      node = cl;
    } else if (vr) {
      node = cr;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return false;
}

// geometric unit normal at p on primitive i
__device__ __forceinline__ f3 prim_normal(const float4* __restrict__ prims, int i, f3 p) {
  const float4* q = prims + 4 * i;
  const int type = __float_as_int(q[0].w) & 3;
  if (type == PRIM_SPHERE) return (p - xyz(q[0])) * q[1].y;
  return xyz(q[3]);
}
__device__ __forceinline__ int prim_material(const float4* __restrict__ prims, int i) {
  return __float_as_int(prims[4 * i].w) >> 2;
}

// ------------------------------------------------------------------ frames
// orthonormal basis around n (Duff et al., JCGT 2017)
struct Frame {
  f3 b1, b2, n;
  __device__ __forceinline__ f3 to_local(f3 w) const { return mk3(dot(w, b1), dot(w, b2), dot(w, n)); }
  __device__ __forceinline__ f3 to_world(f3 l) const { return b1 * l.x + b2 * l.y + n * l.z; }
};
__device__ __forceinline__ Frame make_frame(f3 n) {
  const float sign = copysignf(1.0f, n.z);
  const float a = -1.0f / (sign + n.z);
  const float b = n.x * n.y * a;
  Frame f;
  f.b1 = mk3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  f.b2 = mk3(b, sign + n.y * n.y * a, -n.y);
  f.n = n;
  return f;
}

// ------------------------------------------------------------------- BSDFs
// Lambert (albedo / pi, cosine-weighted sampling) and GGX microfacet
// reflection (Walter et al. 2007): D with roughness alpha, height-correlated
// Smith masking, Schlick Fresnel with F0 = colour, sampling of D(h) cos(theta_h).
constexpr float PI_F = 3.14159265358979323846f;
constexpr float INV_PI_F = 0.318309886183790671538f;
constexpr float TWO_PI_F = 6.28318530717958647692f;

struct Mat {
  int type;
  float alpha;
  f3 col;
};

// Smith Lambda of a unit direction w (local frame): tan^2 = (x^2 + y^2) / z^2,
// written without the cancellation of 1 - cos^2 in float32
__device__ __forceinline__ float ggx_lambda(float a2, f3 w) {
  const float t2 = (w.x * w.x + w.y * w.y) / (w.z * w.z);
  return 0.5f * (-1.0f + sqrtf(1.0f + a2 * t2));
}

// f(wo, wi) |cos theta_i| and the BSDF sampling density (local frame)
__device__ __forceinline__ f3 bsdf_eval(const Mat& m, f3 wo, f3 wi, float& pdf) {
  pdf = 0.0f;
  if (wo.z <= 0.0f || wi.z <= 0.0f) return mk3(0.f, 0.f, 0.f);
  if (m.type == 0) {
    // cos / pi, with one multiplication by 1 / pi instead of divisions
    const float cp = wi.z * INV_PI_F;
    pdf = cp;
    return mk3(m.col.x * cp, m.col.y * cp, m.col.z * cp);
  }
  const float a2 = m.alpha * m.alpha;
  const f3 h = normalize(wo + wi);
  const float woh = dot(wo, h);
  if (woh <= 0.0f) return mk3(0.f, 0.f, 0.f);
  // 1 + cos^2(alpha^2 - 1) = sin^2 + alpha^2 cos^2 for a unit h: no cancellation
  // near the specular peak of a smooth surface
  const float k = (h.x * h.x + h.y * h.y) + a2 * (h.z * h.z);
  const float D = a2 * INV_PI_F / (k * k);
  const float G = 1.0f / (1.0f + ggx_lambda(a2, wo) + ggx_lambda(a2, wi));
  const float sf = 1.0f - woh;
  const float s5 = sf * sf * sf * sf * sf;
  const float D4 = 0.25f * D;
  const float base = D4 * G / wo.z;
  pdf = D4 * h.z / woh;
  return mk3((m.col.x + (1.0f - m.col.x) * s5) * base, (m.col.y + (1.0f - m.col.y) * s5) * base,
             (m.col.z + (1.0f - m.col.z) * s5) * base);
}

__device__ __forceinline__ bool bsdf_sample(const Mat& m, f3 wo, float u0, float u1, f3& wi) {
  if (m.type == 0) {
    const float r = sqrtf(u0);
    float sp, cp;
    sincospif(2.0f * u1, &sp, &cp);   // sin, cos of 2 pi u1 (2 u1 is exact)
    const float z = 1.0f - u0;
    wi = mk3(r * cp, r * sp, sqrtf(z > 0.0f ? z : 0.0f));
    return wi.z > 0.0f;
  }
  const float a2 = m.alpha * m.alpha;
  const float t2 = a2 * u0 / (1.0f - u0);
  const float ct = 1.0f / sqrtf(1.0f + t2);
  const float st = sqrtf(t2) * ct;
  float sp, cp;
  sincospif(2.0f * u1, &sp, &cp);   // sin, cos of 2 pi u1 (2 u1 is exact)
  const f3 h = mk3(st * cp, st * sp, ct);
  const float woh = dot(wo, h);
  if (woh <= 0.0f) return false;
  wi = h * (2.0f * woh) - wo;
  return wi.z > 0.0f;
}

// ------------------------------------------------------------------- guide
// Per-cell directional histogram over (cos theta, phi) in world space: 16 x 16
// equal-area bins.  The bin of a direction is decided in float32.
__device__ __forceinline__ int guide_bin(f3 w) {
  int iz = (int)floorf((w.z + 1.0f) * 8.0f);
  iz = iz < 0 ? 0 : (iz > 15 ? 15 : iz);
  float ph = atan2f(w.y, w.x);
  if (ph < 0.0f) ph += TWO_PI_F;
  int ip = (int)floorf(ph * 2.5464790894703255f);
  ip = ip < 0 ? 0 : (ip > 15 ? 15 : ip);
  return iz * 16 + ip;
}
__device__ __forceinline__ float guide_bin_prob(const float* __restrict__ cdf, int b) {
  return __ldg(cdf + b) - (b > 0 ? __ldg(cdf + b - 1) : 0.0f);
}
__device__ __forceinline__ float guide_pdf(const float* __restrict__ cdf, f3 w) {
  return guide_bin_prob(cdf, guide_bin(w)) * (GUIDE_BINS / (4.0f * PI_F));
}
// First bin b with u < cdf[b] (the last bin if none).  The CDF is
// non-decreasing, so that bin is the number of bins with cdf[b] <= u: count the
// 16 row ends (16 independent loads), then the 16 bins of the row they select
// (four float4 loads) -- two dependent memory round trips instead of the eight
// of a binary search, with the same result.
__device__ __forceinline__ int guide_pick(const float* __restrict__ cdf, float u) {
  float ends[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) ends[k] = __ldg(cdf + 16 * k + 15);
  int row = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) row += ends[k] <= u;
  if (row >= 16) return GUIDE_BINS - 1;
  const float4* r4 = reinterpret_cast<const float4*>(cdf + 16 * row);
  const float4 a = __ldg(r4), b = __ldg(r4 + 1), c = __ldg(r4 + 2), d = __ldg(r4 + 3);
  const int col = (a.x <= u) + (a.y <= u) + (a.z <= u) + (a.w <= u) + (b.x <= u) + (b.y <= u) + (b.z <= u) +
                  (b.w <= u) + (c.x <= u) + (c.y <= u) + (c.z <= u) + (c.w <= u) + (d.x <= u) + (d.y <= u) +
                  (d.z <= u) + (d.w <= u);
  return 16 * row + (col < 16 ? col : 15);
}
__device__ __forceinline__ f3 guide_dir(int b, float u1, float u2) {
  const int iz = b >> 4, ip = b & 15;
  const float z = -1.0f + 2.0f * ((float)iz + u1) / 16.0f;
  float s = (1.0f - z) * (1.0f + z);  // 1 - z^2 without cancellation near the poles
  s = sqrtf(s > 0.0f ? s : 0.0f);
  float sp, cp;
  sincospif(((float)ip + u2) * 0.125f, &sp, &cp);   // phi = 2 pi (ip + u2) / 16
  return mk3(s * cp, s * sp, z);
}

// ----------------------------------------------------------------- counts
// Budgets beta_t of the techniques at a vertex (Sec. 3.1 "Optimization", in the
// spatial form of Sec. 4.1): per channel T_ch / I_ch x q_ch for the RR and the
// splitting factor, their root mean square over the channels ("Handling
// colors"), the three cases (RR below 1, else splitting above 1, else 1) and
// the clamp.  A technique without learned statistics draws its base count:
// NEE 1, the light connection (slot 2 with MARS_TECH_LIGHT) 1, and one
// continuation sample split over the continuation techniques (base_cont: 1
// for BSDF alone, 1/2 each for BSDF and guided).  Then the path multiplicity
// cap b <= max(clamp_lo, M / mult).  on_mask: bit t set if technique t is
// drawn at this vertex.
__device__ __forceinline__ void vertex_budgets(const DevCache& c, const IterArgs& it, int cell, f3 T, float4 est,
                                               float mult, unsigned on_mask, float base_cont, float base2,
                                               float beta[NT]) {
  const float inf = __int_as_float(0x7f800000);
  const f3 f = mk3(T.x / est.x, T.y / est.y, T.z / est.z);
  const float cap = it.max_mult > 0.0f ? fmaxf(it.max_mult / mult, it.clamp_lo) : inf;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const bool on = (on_mask >> t) & 1u;
    float b = on ? (t == 1 ? 1.0f : (t == 2 ? base2 : base_cont)) : 0.0f;
    if (on && it.mode == MARS_MODE_MARS) {
      // both records in one round trip (the second is not worth a dependent load)
      const float4 qr = __ldg(c.cnt + (2 * (NT * cell + t)));
      const float4 qs = __ldg(c.cnt + (2 * (NT * cell + t) + 1));
      if (qr.w > 0.0f) {
        const f3 ar = mul(f, xyz(qr)), as = mul(f, xyz(qs));
        // root mean square over the channels
        const float brr = sqrtf(dot(ar, ar) * (1.0f / 3.0f)), bs = sqrtf(dot(as, as) * (1.0f / 3.0f));
        b = brr < 1.0f ? brr : (bs > 1.0f ? bs : 1.0f);
        b = fminf(fmaxf(b, it.clamp_lo), it.clamp_hi);
      }
    }
    // path multiplicity cap: b <= max(clamp_lo, M / P)
    if (on) b = fminf(b, cap);
    beta[t] = b;
  }
}

// the largest of the three channels
__device__ __forceinline__ float max_channel(f3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }

// ----------------------------------------------------------------- cells
// cell coordinates of a point on an N^3 grid over the scene box; decided in
// float32 like every integer choice, with IEEE round-to-nearest division and
// product whatever the translation unit's division flags
__device__ __forceinline__ void cell_coords(const DevScene& s, int N, f3 p, int idx[3]) {
  const float pa[3] = {p.x, p.y, p.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float f = __fmul_rn(__fdiv_rn(__fsub_rn(pa[a], s.lo[a]), s.ext[a]), (float)N);
    int i = (int)floorf(f);
    idx[a] = i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
  }
}

// uniform grid cell of a point
__device__ __forceinline__ int cell_of(const DevScene& s, int N, f3 p) {
  int idx[3];
  cell_coords(s, N, p, idx);
  return (idx[2] * N + idx[1]) * N + idx[0];
}

// adaptive octree leaf of a point: descend with the bits of its coordinates on
// the finest (2^OCT_LMAX per axis) grid, most significant first.  Scaling by a
// power of two is exact, so an unrefined octree gives the uniform grid's cell.
__device__ __forceinline__ int octree_cell(const DevScene& s, const int* __restrict__ nodes, f3 p) {
  int idx[3];
  cell_coords(s, 1 << OCT_LMAX, p, idx);
  int v = __ldg(nodes);
  for (int level = 0; level < OCT_LMAX && v >= 0; ++level) {
    const int sh = OCT_LMAX - 1 - level;
    const int oct = ((idx[0] >> sh) & 1) | (((idx[1] >> sh) & 1) << 1) | (((idx[2] >> sh) & 1) << 2);
    v = __ldg(nodes + v + oct);
  }
  return ~v;
}

}  // namespace mars
