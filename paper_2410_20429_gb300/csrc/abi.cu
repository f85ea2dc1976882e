// abi.cu -- the C ABI of libmars: scene and cache objects, the per-iteration
// orchestration (pixel tiles over one queue arena), state transfer and the
// error convention (status codes plus a thread-local message).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "abi_internal.h"

namespace mars {

thread_local std::string g_last_error;

// testing hook: countdowns of injected failures (see mars_debug_inject_failure)
static std::atomic<int> g_inject_alloc{0}, g_inject_launch{0};

// true when this call is the one the countdown was set to fail
static bool inject_hit(std::atomic<int>& c) {
  int v = c.load();
  while (v > 0)
    if (c.compare_exchange_weak(v, v - 1)) return v == 1;
  return false;
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st) {
  if (inject_hit(g_inject_alloc)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  static std::once_flag once[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64)
    std::call_once(once[dev], [dev] {
      // keep memory released to the pool instead of returning it to the driver
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    });
  *p = nullptr;
  return cudaMallocAsync(p, bytes, st);
}

void dev_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

namespace {
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;
}  // namespace

void* pinned_acquire(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned_free.lower_bound(bytes);
    if (it != g_pinned_free.end() && it->first <= 2 * bytes) {
      void* p = it->second;
      g_pinned_free.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void pinned_release(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.emplace(bytes, p);
}

mars_status set_error(mars_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

double dlen(const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }
void dcross(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

float host_i2f(int v) {
  float f;
  std::memcpy(&f, &v, sizeof(f));
  return f;
}

int num_sms_of(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 132;
  return n;
}

}  // namespace

// ------------------------------------------------------------------ scene
mars_status scene_create_impl(const mars_scene_desc* d, cudaStream_t st, mars_scene** out) {
  NvtxRange nvtx("mars:scene_create");
  if (!d || !out) return set_error(MARS_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  if (d->n_quads < 0 || d->n_spheres < 0 || d->n_tris < 0 || d->n_materials <= 0)
    return set_error(MARS_ERR_INVALID_ARG, "negative primitive count or no materials");
  const int n = d->n_quads + d->n_spheres + d->n_tris;
  if (n <= 0) return set_error(MARS_ERR_INVALID_ARG, "scene has no primitives");
  if (d->width <= 0 || d->height <= 0 || (int64_t)d->width * d->height > (1ll << 31))
    return set_error(MARS_ERR_INVALID_ARG, "bad resolution %d x %d", d->width, d->height);
  if (d->bvh != MARS_BVH_SAH && d->bvh != MARS_BVH_LBVH)
    return set_error(MARS_ERR_INVALID_ARG, "unknown bvh kind %d", d->bvh);
  if ((d->n_quads && (!d->quads || !d->quad_mat)) || (d->n_spheres && (!d->spheres || !d->sphere_mat)) ||
      (d->n_tris && (!d->tris || !d->tri_mat)) || !d->materials)
    return set_error(MARS_ERR_INVALID_ARG, "null primitive array");
  auto mat_ok = [&](int m) { return m >= 0 && m < d->n_materials; };
  auto emits = [&](int m) {
    const double* r = d->materials + 8 * m;
    return (r[5] + r[6] + r[7]) / 3.0 > 0.0;
  };
  for (int i = 0; i < d->n_materials; ++i) {
    const double* r = d->materials + 8 * i;
    if (!(r[0] == 0.0 || r[0] == 1.0)) return set_error(MARS_ERR_INVALID_ARG, "material %d: bad type", i);
    if (r[0] == 1.0 && !(r[4] > 0.0)) return set_error(MARS_ERR_INVALID_ARG, "material %d: alpha <= 0", i);
  }
  for (int i = 0; i < d->n_quads; ++i)
    if (!mat_ok(d->quad_mat[i])) return set_error(MARS_ERR_INVALID_ARG, "quad %d: material out of range", i);
  for (int i = 0; i < d->n_spheres; ++i) {
    if (!mat_ok(d->sphere_mat[i])) return set_error(MARS_ERR_INVALID_ARG, "sphere %d: material out of range", i);
    if (emits(d->sphere_mat[i])) return set_error(MARS_ERR_INVALID_ARG, "sphere %d: only quads may emit", i);
    if (!(d->spheres[4 * i + 3] > 0.0)) return set_error(MARS_ERR_INVALID_ARG, "sphere %d: radius <= 0", i);
  }
  for (int i = 0; i < d->n_tris; ++i) {
    if (!mat_ok(d->tri_mat[i])) return set_error(MARS_ERR_INVALID_ARG, "triangle %d: material out of range", i);
    if (emits(d->tri_mat[i])) return set_error(MARS_ERR_INVALID_ARG, "triangle %d: only quads may emit", i);
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(MARS_ERR_CUDA, "no CUDA device");
  mars_scene* s = new mars_scene();
  s->device = dev;
  s->stream = st;
  s->num_sms = num_sms_of(dev);
  s->width = d->width;
  s->height = d->height;
  s->n_prims = n;
  s->desc_copy.assign(d);

  // bounds in float64 (primitive corners, sphere boxes, triangle vertices)
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  auto grow = [&](double x, double y, double z) {
    const double p[3] = {x, y, z};
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p[a]);
      hi[a] = std::max(hi[a], p[a]);
    }
  };
  std::vector<float4> prims(4 * (size_t)n), boxes(2 * (size_t)n);
  std::vector<double> blo(3 * (size_t)n), bhi(3 * (size_t)n);
  for (int i = 0; i < d->n_quads; ++i) {
    const double* q = d->quads + 9 * i;
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
      const double c0 = q[a], c1 = q[a] + q[3 + a], c2 = q[a] + q[6 + a], c3 = q[a] + q[3 + a] + q[6 + a];
      mn[a] = std::min(std::min(c0, c1), std::min(c2, c3));
      mx[a] = std::max(std::max(c0, c1), std::max(c2, c3));
    }
    grow(q[0], q[1], q[2]);
    grow(q[0] + q[3], q[1] + q[4], q[2] + q[5]);
    grow(q[0] + q[6], q[1] + q[7], q[2] + q[8]);
    grow(q[0] + q[3] + q[6], q[1] + q[4] + q[7], q[2] + q[5] + q[8]);
    for (int a = 0; a < 3; ++a) { blo[3 * i + a] = mn[a]; bhi[3 * i + a] = mx[a]; }
  }
  for (int k = 0; k < d->n_spheres; ++k) {
    const double* sp = d->spheres + 4 * k;
    const int i = d->n_quads + k;
    grow(sp[0] - sp[3], sp[1] - sp[3], sp[2] - sp[3]);
    grow(sp[0] + sp[3], sp[1] + sp[3], sp[2] + sp[3]);
    for (int a = 0; a < 3; ++a) { blo[3 * i + a] = sp[a] - sp[3]; bhi[3 * i + a] = sp[a] + sp[3]; }
  }
  for (int k = 0; k < d->n_tris; ++k) {
    const double* v = d->tris + 9 * k;
    const int i = d->n_quads + d->n_spheres + k;
    for (int a = 0; a < 3; ++a) {
      blo[3 * i + a] = std::min(std::min(v[a], v[3 + a]), v[6 + a]);
      bhi[3 * i + a] = std::max(std::max(v[a], v[3 + a]), v[6 + a]);
    }
    for (int c = 0; c < 3; ++c) grow(v[3 * c], v[3 * c + 1], v[3 * c + 2]);
  }
  double emax = 0.0;
  for (int a = 0; a < 3; ++a) {
    s->ds.lo[a] = (float)lo[a];
    const double e = hi[a] - lo[a];
    s->ds.ext[a] = (float)(e > 0.0 ? e : 1.0);
    emax = std::max(emax, e);
  }
  // ray offset: 1e-4 x the largest scene extent
  s->ds.eps = (float)(1e-4 * (emax > 0.0 ? emax : 1.0));
  const double pad = 1e-6 * (emax > 0.0 ? emax : 1.0);
  for (int i = 0; i < n; ++i) {
    boxes[2 * i] = make_float4((float)(blo[3 * i] - pad), (float)(blo[3 * i + 1] - pad), (float)(blo[3 * i + 2] - pad), 0.f);
    boxes[2 * i + 1] = make_float4((float)(bhi[3 * i] + pad), (float)(bhi[3 * i + 1] + pad), (float)(bhi[3 * i + 2] + pad), 0.f);
  }

  // lights: emitting quads, picked with probability ~ area x mean radiance
  std::vector<int> light_of_quad(d->n_quads, -1);
  std::vector<double> lw;
  std::vector<int> lq;
  double tot = 0.0;
  for (int i = 0; i < d->n_quads; ++i) {
    const int m = d->quad_mat[i];
    const double* r = d->materials + 8 * m;
    const double p = (r[5] + r[6] + r[7]) / 3.0;
    if (p > 0.0) {
      const double* q = d->quads + 9 * i;
      double nrm[3];
      dcross(q + 3, q + 6, nrm);
      light_of_quad[i] = (int)lq.size();
      lq.push_back(i);
      lw.push_back(dlen(nrm) * p);
      tot += dlen(nrm) * p;
    }
  }
  s->n_lights = (int)lq.size();
  std::vector<float4> lights(5 * std::max<size_t>(1, lq.size()));
  double run = 0.0;
  for (size_t l = 0; l < lq.size(); ++l) {
    const double* q = d->quads + 9 * lq[l];
    const double* r = d->materials + 8 * d->quad_mat[lq[l]];
    double nrm[3];
    dcross(q + 3, q + 6, nrm);
    const double area = dlen(nrm);
    run += lw[l];
    lights[5 * l + 0] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)(run / tot));
    lights[5 * l + 1] = make_float4((float)q[3], (float)q[4], (float)q[5], (float)(lw[l] / tot));
    lights[5 * l + 2] = make_float4((float)q[6], (float)q[7], (float)q[8], (float)area);
    lights[5 * l + 3] = make_float4((float)(nrm[0] / area), (float)(nrm[1] / area), (float)(nrm[2] / area),
                                    host_i2f(lq[l]));
    lights[5 * l + 4] = make_float4((float)r[5], (float)r[6], (float)r[7], 0.f);
  }

  for (int i = 0; i < d->n_quads; ++i) {
    const double* q = d->quads + 9 * i;
    double nrm[3];
    dcross(q + 3, q + 6, nrm);
    const double L = dlen(nrm);
    const int bits = (d->quad_mat[i] << 2) | PRIM_QUAD;
    prims[4 * i + 0] = make_float4((float)q[0], (float)q[1], (float)q[2], host_i2f(bits));
    prims[4 * i + 1] = make_float4((float)q[3], (float)q[4], (float)q[5], 0.f);
    prims[4 * i + 2] = make_float4((float)q[6], (float)q[7], (float)q[8], 0.f);
    prims[4 * i + 3] = make_float4((float)(nrm[0] / L), (float)(nrm[1] / L), (float)(nrm[2] / L),
                                   host_i2f(light_of_quad[i]));
  }
  for (int k = 0; k < d->n_spheres; ++k) {
    const double* sp = d->spheres + 4 * k;
    const int i = d->n_quads + k;
    const int bits = (d->sphere_mat[k] << 2) | PRIM_SPHERE;
    prims[4 * i + 0] = make_float4((float)sp[0], (float)sp[1], (float)sp[2], host_i2f(bits));
    prims[4 * i + 1] = make_float4((float)sp[3], (float)(1.0 / sp[3]), 0.f, 0.f);
    prims[4 * i + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    prims[4 * i + 3] = make_float4(0.f, 0.f, 0.f, host_i2f(-1));
  }
  for (int k = 0; k < d->n_tris; ++k) {
    const double* v = d->tris + 9 * k;
    const int i = d->n_quads + d->n_spheres + k;
    const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    const double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    double nrm[3];
    dcross(e1, e2, nrm);
    const double L = dlen(nrm);
    const int bits = (d->tri_mat[k] << 2) | PRIM_TRI;
    prims[4 * i + 0] = make_float4((float)v[0], (float)v[1], (float)v[2], host_i2f(bits));
    prims[4 * i + 1] = make_float4((float)e1[0], (float)e1[1], (float)e1[2], 0.f);
    prims[4 * i + 2] = make_float4((float)e2[0], (float)e2[1], (float)e2[2], 0.f);
    prims[4 * i + 3] = make_float4((float)(nrm[0] / L), (float)(nrm[1] / L), (float)(nrm[2] / L), host_i2f(-1));
  }
  std::vector<float4> mats(3 * (size_t)d->n_materials);
  for (int m = 0; m < d->n_materials; ++m) {
    const double* r = d->materials + 8 * m;
    const bool refl = r[1] > 0.0 || r[2] > 0.0 || r[3] > 0.0;
    mats[3 * m + 0] = make_float4((float)r[0], (float)r[4], refl ? 1.f : 0.f, emits(m) ? 1.f : 0.f);
    mats[3 * m + 1] = make_float4((float)r[1], (float)r[2], (float)r[3], 0.f);
    mats[3 * m + 2] = make_float4((float)r[5], (float)r[6], (float)r[7], 0.f);
  }
  // pinhole camera: right = normalize(up x forward), true up = forward x right
  {
    const double* c = d->camera;
    double f[3] = {c[3] - c[0], c[4] - c[1], c[5] - c[2]};
    const double fl = dlen(f);
    for (double& x : f) x /= fl;
    double r[3];
    dcross(c + 6, f, r);
    const double rl = dlen(r);
    for (double& x : r) x /= rl;
    double u[3];
    dcross(f, r, u);
    for (int a = 0; a < 3; ++a) {
      s->ds.cam_o[a] = (float)c[a];
      s->ds.cam_f[a] = (float)f[a];
      s->ds.cam_r[a] = (float)r[a];
      s->ds.cam_u[a] = (float)u[a];
    }
    s->ds.tanh_half = (float)std::tan(0.5 * c[9] * 3.14159265358979323846 / 180.0);
    s->ds.aspect = (float)((double)d->width / (double)d->height);
  }
  s->ds.n_prims = n;
  s->ds.n_quads = d->n_quads;
  s->ds.n_lights = s->n_lights;
  s->ds.n_mats = d->n_materials;
  s->ds.width = d->width;
  s->ds.height = d->height;

  auto cleanup = [&](cudaError_t e, const char* what) {
    set_error(e == cudaErrorMemoryAllocation ? MARS_ERR_OOM : MARS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    scene_destroy_impl(s);
    return e == cudaErrorMemoryAllocation ? MARS_ERR_OOM : MARS_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = dev_alloc((void**)&s->d_prims, sizeof(float4) * prims.size(), st)) != cudaSuccess) return cleanup(e, "scene alloc");
  if ((e = dev_alloc((void**)&s->d_boxes, sizeof(float4) * boxes.size(), st)) != cudaSuccess) return cleanup(e, "scene alloc");
  if ((e = dev_alloc((void**)&s->d_nodes, sizeof(BvhNode) * std::max(1, n - 1), st)) != cudaSuccess) return cleanup(e, "scene alloc");
  if ((e = dev_alloc((void**)&s->d_mats, sizeof(float4) * mats.size(), st)) != cudaSuccess) return cleanup(e, "scene alloc");
  if ((e = dev_alloc((void**)&s->d_lights, sizeof(float4) * lights.size(), st)) != cudaSuccess) return cleanup(e, "scene alloc");
  if ((e = cudaMemcpyAsync(s->d_prims, prims.data(), sizeof(float4) * prims.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(s->d_boxes, boxes.data(), sizeof(float4) * boxes.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(s->d_mats, mats.data(), sizeof(float4) * mats.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(s->d_lights, lights.data(), sizeof(float4) * lights.size(), cudaMemcpyHostToDevice, st)))
    return cleanup(e, "scene upload");
  NvtxRange nvtx_bvh("mars:bvh_build");
  if (d->bvh == MARS_BVH_SAH && n >= 2) {
    std::vector<BvhNode> sah;
    if (!build_bvh_sah(boxes, n, sah)) {
      set_error(MARS_ERR_CUDA, "SAH build produced an invalid hierarchy");
      scene_destroy_impl(s);
      return MARS_ERR_CUDA;
    }
    if ((e = cudaMemcpyAsync(s->d_nodes, sah.data(), sizeof(BvhNode) * (n - 1), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return cleanup(e, "BVH upload");
  } else {
    std::string berr;
    if ((e = build_bvh(s->d_boxes, n, s->ds.lo, s->ds.ext, s->d_nodes, st, &berr)) != cudaSuccess)
      return cleanup(e, berr.c_str());
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cleanup(e, "scene create");
  if (n >= 2) {
    // check the hierarchy before any kernel traverses it: every internal node
    // reached once from the root, every primitive once, all indices in range
    std::vector<BvhNode> nodes(n - 1);
    if ((e = cudaMemcpyAsync(nodes.data(), s->d_nodes, sizeof(BvhNode) * (n - 1), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cleanup(e, "BVH readback");
    std::vector<uint8_t> seen_node(n - 1, 0), seen_leaf(n, 0);
    std::vector<int> stack{0};
    bool okb = true;
    while (!stack.empty() && okb) {
      const int k = stack.back();
      stack.pop_back();
      if (k < 0 || k >= n - 1 || seen_node[k]) { okb = false; break; }
      seen_node[k] = 1;
      int ch[2];
      std::memcpy(&ch[0], &nodes[k].a.w, sizeof(int));
      std::memcpy(&ch[1], &nodes[k].b.w, sizeof(int));
      for (int c : ch) {
        if (c < 0) {
          const int leaf = ~c;
          if (leaf >= n || seen_leaf[leaf]) { okb = false; break; }
          seen_leaf[leaf] = 1;
        } else {
          stack.push_back(c);
        }
      }
    }
    for (int k = 0; okb && k < n - 1; ++k) okb = seen_node[k];
    for (int k = 0; okb && k < n; ++k) okb = seen_leaf[k];
    if (!okb) {
      set_error(MARS_ERR_CUDA, "BVH build produced an invalid hierarchy");
      scene_destroy_impl(s);
      return MARS_ERR_CUDA;
    }
  }
  if (n >= 2) {
    // collapse the binary hierarchy into 4-wide nodes: a node's children are
    // grown by replacing the internal child with the largest box surface by its
    // two children until there are four or only leaves remain
    std::vector<BvhNode> bin(n - 1);
    if ((e = cudaMemcpyAsync(bin.data(), s->d_nodes, sizeof(BvhNode) * (n - 1), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cleanup(e, "BVH readback");
    struct Ch {
      int id;              // >= 0 binary internal node, < 0 ~primitive
      float lo[3], hi[3];
    };
    auto kids = [&](int k, Ch out[2]) {
      const BvhNode& b = bin[k];
      int l, r;
      std::memcpy(&l, &b.a.w, sizeof(int));
      std::memcpy(&r, &b.b.w, sizeof(int));
      out[0] = {l, {b.a.x, b.a.y, b.a.z}, {b.b.x, b.b.y, b.b.z}};
      out[1] = {r, {b.c.x, b.c.y, b.c.z}, {b.d.x, b.d.y, b.d.z}};
    };
    auto area = [](const Ch& c) {
      const double dx = c.hi[0] - c.lo[0], dy = c.hi[1] - c.lo[1], dz = c.hi[2] - c.lo[2];
      return dx * dy + dy * dz + dz * dx;
    };
    std::vector<Bvh4Node> n4;
    n4.reserve(n);
    std::vector<std::pair<int, int>> todo;  // (binary node, BVH4 slot)
    n4.emplace_back();
    todo.emplace_back(0, 0);
    while (!todo.empty()) {
      const auto [bk, slot] = todo.back();
      todo.pop_back();
      Ch set[4];
      int m = 2;
      kids(bk, set);
      while (m < 4) {
        int best = -1;
        double ba = -1.0;
        for (int k = 0; k < m; ++k)
          if (set[k].id >= 0 && area(set[k]) > ba) { ba = area(set[k]); best = k; }
        if (best < 0) break;
        Ch two[2];
        kids(set[best].id, two);
        set[best] = two[0];
        set[m++] = two[1];
      }
      float lo[3][4], hi[3][4];
      int ch[4];
      for (int k = 0; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) {
          lo[a][k] = k < m ? set[k].lo[a] : 0.0f;   // empty slot (child BVH4_EMPTY): never visited
          hi[a][k] = k < m ? set[k].hi[a] : 0.0f;
        }
        if (k >= m) {
          ch[k] = BVH4_EMPTY;
        } else if (set[k].id < 0) {
          ch[k] = set[k].id;
        } else {
          ch[k] = (int)n4.size();
          n4.emplace_back();
          todo.emplace_back(set[k].id, ch[k]);
        }
      }
      Bvh4Node& nd = n4[slot];
      nd.lox = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
      nd.loy = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
      nd.loz = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
      nd.hix = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
      nd.hiy = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
      nd.hiz = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
      nd.child = make_int4(ch[0], ch[1], ch[2], ch[3]);
      nd.pad = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if ((e = dev_alloc((void**)&s->d_nodes4, sizeof(Bvh4Node) * n4.size(), st)) != cudaSuccess)
      return cleanup(e, "scene alloc");
    if ((e = cudaMemcpyAsync(s->d_nodes4, n4.data(), sizeof(Bvh4Node) * n4.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cleanup(e, "BVH4 upload");
    s->ds.n_nodes4 = (int)n4.size();
  }
  s->ds.nodes4 = s->d_nodes4;
  s->ds.prims = s->d_prims;
  s->ds.nodes = s->d_nodes;
  s->ds.mats = s->d_mats;
  s->ds.lights = s->d_lights;
  s->device_bytes = sizeof(float4) * (prims.size() + boxes.size() + mats.size() + lights.size()) +
                    sizeof(BvhNode) * std::max(1, n - 1);
  *out = s;
  return MARS_OK;
}

void scene_destroy_impl(mars_scene* s) {
  if (!s) return;
  DeviceGuard g(s->device);
  // the scene's last users are the caches' iterations, which end synchronised;
  // release on its creation stream
  cudaStream_t st = s->stream;
  if (cudaStreamQuery(st) == cudaErrorInvalidResourceHandle) st = cudaStreamPerThread;
  dev_free(s->d_prims, st);
  dev_free(s->d_boxes, st);
  dev_free(s->d_nodes, st);
  dev_free(s->d_nodes4, st);
  dev_free(s->d_mats, st);
  dev_free(s->d_lights, st);
  delete s;
}

// ------------------------------------------------------------------ cache
// images below this size render in one lane (two half tiles measured 2 %
// slower at 128 x 128 and 1.5 % at 256 x 256, 5 % faster at 512 x 512); above
// it, one lane per 2^16 pixels up to the cache's lanes
constexpr int64_t kLaneMinPixels = 1 << 17;
constexpr int kDefaultLanes = 2;
constexpr int64_t kLaneFloorPixels = 1 << 14;  // the autotuner tries lanes on images from this size

uint64_t cache_footprint(int64_t cells, int64_t pixels, int max_depth, int techniques, uint64_t cap) {
  (void)max_depth;
  uint64_t b = (uint64_t)cap * (SLOT_BYTES + SHADOW_BYTES);
  if (techniques & MARS_TECH_LIGHT) b += (uint64_t)cap * LIGHT_SLOT_BYTES;
  b += (uint64_t)cells * NT * (2 * sizeof(float4) + NSTAT * sizeof(double));
  if (techniques & MARS_TECH_GUIDED) b += (uint64_t)cells * GUIDE_BINS * 2 * sizeof(float);
  b += (uint64_t)pixels * 4 * sizeof(float4);  // running sum, estimate, image, combination
  b += (uint64_t)IMG_TOPK_BLOCKS * MAX_DROP * sizeof(unsigned long long);
  return b + sizeof(DevCounters) + 4096 * (sizeof(IterArgs) + sizeof(unsigned int)) + 4096;
}

uint64_t default_capacity(int64_t pixels, int max_depth) {
  // a MARS iteration of the guided room at 512^2 holds about 1.4 x pixels x D
  // rays; heavier splitting that overflows this falls back to pixel tiles
  uint64_t cap = (uint64_t)pixels * (uint64_t)max_depth * 3ull;
  if (cap < (1ull << 20)) cap = 1ull << 20;
  return cap;
}

mars_status cache_create_impl(const mars_scene* s, const mars_cache_desc* d, cudaStream_t st, mars_cache** out) {
  NvtxRange nvtx("mars:cache_create");
  if (!s || !d || !out) return set_error(MARS_ERR_INVALID_ARG, "null scene, descriptor or output");
  *out = nullptr;
  if (d->grid_n < 1 || d->grid_n > 256) return set_error(MARS_ERR_INVALID_ARG, "grid_n %d out of [1, 256]", d->grid_n);
  if (!(d->techniques & MARS_TECH_BSDF) || (d->techniques & ~15))
    return set_error(MARS_ERR_INVALID_ARG, "techniques must include BSDF and only use bits 0..3");
  if ((d->techniques & MARS_TECH_GUIDED) && (d->techniques & MARS_TECH_LIGHT))
    return set_error(MARS_ERR_INVALID_ARG, "the guided technique and light connections share slot 2");
  if ((d->techniques & MARS_TECH_LIGHT) && s->n_lights == 0)
    return set_error(MARS_ERR_INVALID_ARG, "light connections requested but the scene has no emitting quad");
  if (d->max_depth < 1 || d->max_depth > MAXD)
    return set_error(MARS_ERR_INVALID_ARG, "max_depth %d out of [1, %d]", d->max_depth, MAXD);
  if ((d->techniques & MARS_TECH_NEE) && s->n_lights == 0)
    return set_error(MARS_ERR_INVALID_ARG, "NEE requested but the scene has no emitting quad");
  if (d->flags & ~(MARS_CACHE_FP32_STATISTICS | MARS_CACHE_OCTREE | MARS_CACHE_NO_GRAPHS | MARS_CACHE_ONE_LANE))
    return set_error(MARS_ERR_INVALID_ARG, "unknown cache flags %d", d->flags);
  const bool fp32 = (d->flags & MARS_CACHE_FP32_STATISTICS) != 0;
  const bool octree = (d->flags & MARS_CACHE_OCTREE) != 0;
  const int bits = (d->techniques & MARS_TECH_GUIDED) ? 6 : 5;
  if ((d->max_depth - 1) * bits > 64)
    return set_error(MARS_ERR_INVALID_ARG, "max_depth %d too deep for %d lineage bits per level", d->max_depth, bits);
  const int64_t grid_cells = (int64_t)d->grid_n * d->grid_n * d->grid_n;
  int64_t cells = grid_cells;
  int oct_levels = 0;
  if (octree) {
    while ((1 << oct_levels) < d->grid_n) ++oct_levels;
    if ((1 << oct_levels) != d->grid_n || oct_levels > OCT_LMAX)
      return set_error(MARS_ERR_INVALID_ARG, "octree: grid_n %d is not a power of two up to %d", d->grid_n,
                       1 << OCT_LMAX);
    const int64_t ml = d->max_leaves ? d->max_leaves : 65536;
    if (ml < grid_cells || ml > (1 << 24))
      return set_error(MARS_ERR_INVALID_ARG, "octree: max_leaves %lld outside [grid_n^3, 2^24]", (long long)ml);
    if (d->split_samples < 0.0f) return set_error(MARS_ERR_INVALID_ARG, "octree: split_samples < 0");
    cells = ml;
  }
  const int64_t pixels = (int64_t)s->width * s->height;
  uint64_t cap = d->arena_capacity ? d->arena_capacity : default_capacity(pixels, d->max_depth);
  if (cap < 64) cap = 64;
  if (cap > 0xFFFFFFF0ull) return set_error(MARS_ERR_INVALID_ARG, "arena_capacity above 2^32 - 16");

  DeviceGuard g(s->device);
  mars_cache* c = new mars_cache();
  c->scene = s;
  c->device = s->device;
  c->last_stream = st;
  c->grid_n = d->grid_n;
  c->techniques = d->techniques;
  c->max_depth = d->max_depth;
  c->cells = cells;
  c->pixels = pixels;
  c->arena.cap = cap;
  c->arena.scap = cap;  // NEE shadow rays: as many slots as rays
  c->arena.lcap = (d->techniques & MARS_TECH_LIGHT) ? cap : 0;  // light connection samples: likewise
  c->arena.vcap = c->arena.lcap;                                  // and light subpath vertices
  c->max_tiles = 4096;
  // two tile lanes (each with half the arena) unless asked for one or the
  // image has a single pixel
  c->lanes = ((d->flags & MARS_CACHE_ONE_LANE) || pixels < 2 || cap < 128) ? 1 : kDefaultLanes;
  c->use_lanes = c->lanes;
  c->lane_min_pixels = kLaneMinPixels;
  auto cleanup = [&](cudaError_t e, const char* what) {
    const mars_status ms = e == cudaErrorMemoryAllocation ? MARS_ERR_OOM : MARS_ERR_CUDA;
    set_error(ms, "%s: %s", what, cudaGetErrorString(e));
    cache_destroy_impl(c);
    return ms;
  };
  cudaError_t e;
  for (int k = 0; k < NR; ++k)
    if ((e = dev_alloc((void**)&c->arena.R[k], sizeof(float4) * cap, st)) != cudaSuccess) return cleanup(e, "arena alloc");
  for (int k = 0; k < NV; ++k)
    if ((e = dev_alloc((void**)&c->arena.V[k], sizeof(float4) * cap, st)) != cudaSuccess) return cleanup(e, "arena alloc");
  if ((e = dev_alloc((void**)&c->arena.S, sizeof(float4) * cap, st)) != cudaSuccess) return cleanup(e, "arena alloc");
  if ((e = dev_alloc((void**)&c->arena.M, sizeof(float) * cap, st)) != cudaSuccess) return cleanup(e, "arena alloc");
  if ((e = dev_alloc((void**)&c->arena.H, sizeof(float2) * cap, st)) != cudaSuccess) return cleanup(e, "arena alloc");
  for (int k = 0; k < NSH; ++k)
    if ((e = dev_alloc((void**)&c->arena.SH[k], sizeof(float4) * c->arena.scap, st)) != cudaSuccess)
      return cleanup(e, "arena alloc");
  if ((e = dev_alloc((void**)&c->arena.SL, sizeof(unsigned int) * c->arena.scap, st)) != cudaSuccess)
    return cleanup(e, "arena alloc");
  if (c->arena.lcap) {
    if ((e = dev_alloc((void**)&c->arena.R5, sizeof(float4) * cap, st)) != cudaSuccess) return cleanup(e, "arena alloc");
    for (int k = 0; k < NLJ; ++k)
      if ((e = dev_alloc((void**)&c->arena.LJ[k], sizeof(float4) * c->arena.lcap, st)) != cudaSuccess)
        return cleanup(e, "arena alloc");
    if ((e = dev_alloc((void**)&c->arena.LR, sizeof(float4) * c->arena.lcap, st)) != cudaSuccess)
      return cleanup(e, "arena alloc");
    for (int k = 0; k < NLV; ++k)
      if ((e = dev_alloc((void**)&c->arena.LV[k], sizeof(float4) * c->arena.vcap, st)) != cudaSuccess)
        return cleanup(e, "arena alloc");
    if ((e = dev_alloc((void**)&c->arena.LC, sizeof(float4) * c->arena.vcap, st)) != cudaSuccess)
      return cleanup(e, "arena alloc");
  }
  if ((e = dev_alloc((void**)&c->d_cnt, sizeof(float4) * 2 * NT * cells, st)) != cudaSuccess) return cleanup(e, "cache alloc");
  c->fp32_stats = fp32;
  if (fp32) {
    if ((e = dev_alloc((void**)&c->d_stats32, sizeof(float) * NSTAT * NT * cells, st)) != cudaSuccess)
      return cleanup(e, "cache alloc");
  } else if ((e = dev_alloc((void**)&c->d_stats, sizeof(double) * NSTAT * NT * cells, st)) != cudaSuccess) {
    return cleanup(e, "cache alloc");
  }
  const int64_t gcells = (d->techniques & MARS_TECH_GUIDED) ? cells : 1;
  if ((e = dev_alloc((void**)&c->d_hist, sizeof(float) * GUIDE_BINS * gcells, st)) != cudaSuccess) return cleanup(e, "cache alloc");
  if ((e = dev_alloc((void**)&c->d_cdf, sizeof(float) * GUIDE_BINS * gcells, st)) != cudaSuccess) return cleanup(e, "cache alloc");
  if ((e = dev_alloc((void**)&c->d_guide_dirty, (size_t)gcells, st)) != cudaSuccess) return cleanup(e, "cache alloc");
  if ((e = dev_alloc((void**)&c->d_est, sizeof(float4) * pixels, st)) != cudaSuccess) return cleanup(e, "image alloc");
  if ((e = dev_alloc((void**)&c->d_run, sizeof(float4) * pixels, st)) != cudaSuccess) return cleanup(e, "image alloc");
  if ((e = dev_alloc((void**)&c->d_img, sizeof(float4) * pixels, st)) != cudaSuccess) return cleanup(e, "image alloc");
  if ((e = dev_alloc((void**)&c->d_ctr, sizeof(DevCounters) * mars_cache::kMaxLanes, st)) != cudaSuccess)
    return cleanup(e, "counter alloc");
  if ((e = dev_alloc((void**)&c->d_tile_status, sizeof(unsigned int) * c->max_tiles, st)) != cudaSuccess)
    return cleanup(e, "counter alloc");
  c->h_ctr = (DevCounters*)pinned_acquire(sizeof(DevCounters));
  if (!c->h_ctr) return cleanup(cudaErrorMemoryAllocation, "pinned alloc");
  c->h_tile_status = (unsigned int*)pinned_acquire(sizeof(unsigned int) * c->max_tiles);
  if (!c->h_tile_status) return cleanup(cudaErrorMemoryAllocation, "pinned alloc");
  if ((e = dev_alloc((void**)&c->d_args, sizeof(IterArgs) * c->max_tiles, st)) != cudaSuccess)
    return cleanup(e, "argument alloc");
  c->h_args = (IterArgs*)pinned_acquire(sizeof(IterArgs) * c->max_tiles);
  if (!c->h_args) return cleanup(cudaErrorMemoryAllocation, "pinned alloc");
  if ((e = dev_alloc((void**)&c->d_comb, sizeof(float4) * pixels, st)) != cudaSuccess ||
      (e = dev_alloc((void**)&c->d_comb_w, sizeof(double), st)) != cudaSuccess ||
      (e = dev_alloc((void**)&c->d_img_acc, 3 * sizeof(double), st)) != cudaSuccess ||
      (e = dev_alloc((void**)&c->d_topk, sizeof(unsigned long long) * IMG_TOPK_BLOCKS * MAX_DROP, st)) !=
          cudaSuccess)
    return cleanup(e, "image alloc");
  cudaMemsetAsync(c->d_comb, 0, sizeof(float4) * pixels, st);
  cudaMemsetAsync(c->d_comb_w, 0, sizeof(double), st);
  cudaMemsetAsync(c->d_img_acc, 0, 3 * sizeof(double), st);
  c->use_graphs = (d->flags & MARS_CACHE_NO_GRAPHS) == 0;
  cudaMemsetAsync(c->d_cnt, 0, sizeof(float4) * 2 * NT * cells, st);
  if (c->d_stats) cudaMemsetAsync(c->d_stats, 0, sizeof(double) * NSTAT * NT * cells, st);
  if (c->d_stats32) cudaMemsetAsync(c->d_stats32, 0, sizeof(float) * NSTAT * NT * cells, st);
  cudaMemsetAsync(c->d_hist, 0, sizeof(float) * GUIDE_BINS * gcells, st);
  cudaMemsetAsync(c->d_guide_dirty, 0, (size_t)gcells, st);
  cudaMemsetAsync(c->d_run, 0, sizeof(float4) * pixels, st);
  cudaMemsetAsync(c->d_img, 0, sizeof(float4) * pixels, st);
  cudaMemsetAsync(c->d_ctr, 0, sizeof(DevCounters) * mars_cache::kMaxLanes, st);
  cudaMemsetAsync(c->d_tile_status, 0, sizeof(unsigned int) * c->max_tiles, st);
  {
    std::vector<float> cdf((size_t)GUIDE_BINS * gcells);
    for (int64_t k = 0; k < gcells; ++k)
      for (int b = 0; b < GUIDE_BINS; ++b) cdf[k * GUIDE_BINS + b] = (float)((double)(b + 1) / GUIDE_BINS);
    std::vector<float4> one((size_t)pixels, make_float4(1.f, 1.f, 1.f, 0.f));
    if ((e = cudaMemcpyAsync(c->d_cdf, cdf.data(), sizeof(float) * cdf.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_est, one.data(), sizeof(float4) * one.size(), cudaMemcpyHostToDevice, st)))
      return cleanup(e, "cache init");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cleanup(e, "cache init");
  }
  c->dc.grid_n = d->grid_n;
  c->dc.n_cells = (int)cells;
  c->dc.techniques = d->techniques;
  c->dc.max_depth = d->max_depth;
  c->dc.bits = bits;
  c->dc.n_pixels = (int)pixels;
  c->dc.cnt = c->d_cnt;
  c->dc.stats = c->d_stats;
  c->dc.stats32 = c->d_stats32;
  c->dc.guide_hist = c->d_hist;
  c->dc.guide_cdf = c->d_cdf;
  c->dc.guide_dirty = c->d_guide_dirty;
  c->dc.est = c->d_est;
  c->dc.run_sum = c->d_run;
  c->dc.img = c->d_img;
  c->dc.ctr = c->d_ctr;
  c->dc.tile_status = c->d_tile_status;
  c->dc.comb = c->d_comb;
  c->dc.comb_w = c->d_comb_w;
  c->dc.img_acc = c->d_img_acc;
  c->dc.topk = c->d_topk;
  if (octree) {
    // the initial tree equals the grid: levels 0..L0 complete, breadth first,
    // children of a node consecutive by octant, leaves numbered like the grid
    const int N = d->grid_n;
    std::vector<int> nodes, level((size_t)cells, 0), lnode((size_t)cells, 0);
    std::vector<int> cur{0, 0, 0}, nxt;
    nodes.push_back(0);
    int first = 0, count = 1;
    for (int l = 0; l <= oct_levels; ++l) {
      nxt.clear();
      const int next_first = first + count;
      for (int k = 0; k < count; ++k) {
        const int x = cur[3 * k], y = cur[3 * k + 1], z = cur[3 * k + 2];
        if (l == oct_levels) {
          const int cell = (z * N + y) * N + x;
          nodes[first + k] = ~cell;
          level[cell] = oct_levels;
          lnode[cell] = first + k;
        } else {
          nodes[first + k] = next_first + 8 * k;
          for (int o = 0; o < 8; ++o) {
            nxt.push_back(2 * x + (o & 1));
            nxt.push_back(2 * y + ((o >> 1) & 1));
            nxt.push_back(2 * z + ((o >> 2) & 1));
          }
        }
      }
      if (l < oct_levels) {
        nodes.resize((size_t)next_first + 8 * count);
        first = next_first;
        count *= 8;
        cur.swap(nxt);
      }
    }
    const int n_nodes = (int)nodes.size();
    const int cap_nodes = n_nodes + 8 * (int)((cells - grid_cells) / 7 + 1);
    const int meta[3] = {n_nodes, (int)grid_cells, 0};
    if ((e = dev_alloc((void**)&c->d_oct_nodes, sizeof(int) * cap_nodes, st)) != cudaSuccess ||
        (e = dev_alloc((void**)&c->d_oct_level, sizeof(int) * cells, st)) != cudaSuccess ||
        (e = dev_alloc((void**)&c->d_oct_lnode, sizeof(int) * cells, st)) != cudaSuccess ||
        (e = dev_alloc((void**)&c->d_oct_meta, sizeof(int) * 4, st)) != cudaSuccess ||
        (e = dev_alloc((void**)&c->d_oct_split, sizeof(int) * (cells / 7 + 1), st)) != cudaSuccess ||
        (e = dev_alloc((void**)&c->d_oct_leaf_n, sizeof(float) * cells, st)) != cudaSuccess)
      return cleanup(e, "octree alloc");
    if ((e = cudaMemcpyAsync(c->d_oct_nodes, nodes.data(), sizeof(int) * n_nodes, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_oct_level, level.data(), sizeof(int) * cells, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_oct_lnode, lnode.data(), sizeof(int) * cells, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_oct_meta, meta, sizeof(int) * 3, cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st)))
      return cleanup(e, "octree init");
    c->oct_cap_nodes = cap_nodes;
    c->dc.oct_nodes = c->d_oct_nodes;
    c->dc.oct_leaf_level = c->d_oct_level;
    c->dc.oct_leaf_node = c->d_oct_lnode;
    c->dc.oct_meta = c->d_oct_meta;
    c->dc.oct_split = c->d_oct_split;
    c->dc.oct_leaf_n = c->d_oct_leaf_n;
    c->dc.oct_cap_nodes = cap_nodes;
    c->dc.split_samples = d->split_samples > 0.0f ? d->split_samples : 4096.0f;
  }
  c->device_bytes = cache_footprint(cells, pixels, d->max_depth, d->techniques, cap);
  const bool light = (d->techniques & MARS_TECH_LIGHT) != 0;
  if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup(e, "side stream");
  if (light && (e = cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup(e, "side stream");
  for (int k = 0; k <= d->max_depth + 1; ++k) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e, "event");
    c->sync_events.push_back(ev);
  }
  if (c->lanes > 1 && (e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming)) != cudaSuccess)
    return cleanup(e, "lane event");
  for (int l = 1; l < c->lanes; ++l) {
    cudaStream_t a = nullptr, b = nullptr;
    cudaEvent_t j = nullptr;
    if ((e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking)) == cudaSuccess) c->lane_st.push_back(a);
    if (e == cudaSuccess && (e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking)) == cudaSuccess)
      c->lane_side.push_back(b);
    if (e == cudaSuccess && light) {
      cudaStream_t b2 = nullptr;
      if ((e = cudaStreamCreateWithFlags(&b2, cudaStreamNonBlocking)) == cudaSuccess) c->lane_side2.push_back(b2);
    }
    if (e == cudaSuccess && (e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) == cudaSuccess)
      c->join_ev.push_back(j);
    if (e != cudaSuccess) return cleanup(e, "lane streams");
    c->lane_sync.emplace_back();
    for (int k = 0; k <= d->max_depth + 1; ++k) {
      cudaEvent_t ev;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cleanup(e, "event");
      c->lane_sync.back().push_back(ev);
    }
  }
  {
    const int threads[WAVE_KERNELS] = {128, 128, 128, 128};
    const int bps[WAVE_KERNELS] = {0, 0, 0, 0};
    const int var[WAVE_KERNELS] = {0, 0, 0, 0};
    const mars_status ls = apply_launch(c, threads, bps, var);
    if (ls != MARS_OK) {
      cache_destroy_impl(c);
      return ls;
    }
  }
  *out = c;
  return MARS_OK;
}

// Grid of each wave kernel = SMs x resident blocks per SM (the occupancy
// maximum unless a positive count is given): a persistent grid that strides
// over the wave.
mars_status apply_launch(mars_cache* c, const int threads[WAVE_KERNELS], const int blocks_per_sm[WAVE_KERNELS],
                         const int variant[WAVE_KERNELS]) {
  for (int k = 0; k < WAVE_KERNELS; ++k) {
    if (variant[k] < 0 || variant[k] >= wave_variants(k))
      return set_error(MARS_ERR_INVALID_ARG, "wave kernel %d: no register-cap variant %d", k, variant[k]);
    if (!wave_threads_ok(threads[k]))
      return set_error(MARS_ERR_INVALID_ARG, "wave kernel %d: %d threads per block (need a multiple of 32 in 32..256)",
                       k, threads[k]);
    if (blocks_per_sm[k] < 0 || blocks_per_sm[k] > 64)
      return set_error(MARS_ERR_INVALID_ARG, "wave kernel %d: blocks per SM %d outside 0..64", k, blocks_per_sm[k]);
  }
  int occ[WAVE_KERNELS];
  const cudaError_t e = wave_occupancy(threads, variant, occ);
  if (e != cudaSuccess) return set_error(MARS_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(e));
  for (int k = 0; k < WAVE_KERNELS; ++k) {
    const int b = blocks_per_sm[k] > 0 ? blocks_per_sm[k] : std::max(1, occ[k]);
    c->launch.threads[k] = threads[k];
    c->launch.variant[k] = variant[k];
    c->launch.grid[k] = c->scene->num_sms * b;
    c->blocks_per_sm[k] = b;
  }
  return MARS_OK;
}

void cache_destroy_impl(mars_cache* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  // work still queued for the cache (an update, a state copy) is on the stream
  // of its last call: let it finish, then release the memory to the pool
  cudaStream_t st = c->last_stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaDeviceSynchronize();
    st = cudaStreamPerThread;
  }
  for (auto* p : c->arena.R) dev_free(p, st);
  for (auto* p : c->arena.V) dev_free(p, st);
  dev_free(c->arena.S, st);
  dev_free(c->arena.M, st);
  dev_free(c->arena.H, st);
  for (auto* p : c->arena.SH) dev_free(p, st);
  dev_free(c->arena.SL, st);
  dev_free(c->arena.R5, st);
  for (auto* p : c->arena.LJ) dev_free(p, st);
  dev_free(c->arena.LR, st);
  for (auto* p : c->arena.LV) dev_free(p, st);
  dev_free(c->arena.LC, st);
  void* ptrs[] = {c->d_cnt, c->d_stats, c->d_stats32, c->d_hist, c->d_cdf, c->d_guide_dirty, c->d_est, c->d_run,
                  c->d_img, c->d_ctr, c->d_tile_status, c->d_oct_nodes, c->d_oct_level, c->d_oct_lnode,
                  c->d_oct_meta, c->d_oct_split, c->d_oct_leaf_n, c->d_comb, c->d_comb_w, c->d_img_acc, c->d_topk};
  for (void* p : ptrs) dev_free(p, st);
  pinned_release(c->h_ctr, sizeof(DevCounters));
  pinned_release(c->h_tile_status, sizeof(unsigned int) * c->max_tiles);
  dev_free(c->d_args, st);
  dev_free(c->d_host_stage, st);
  pinned_release(c->h_args, sizeof(IterArgs) * c->max_tiles);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  for (cudaEvent_t ev : c->events) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c->sync_events) cudaEventDestroy(ev);
  for (auto& v : c->lane_sync)
    for (cudaEvent_t ev : v) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c->join_ev) cudaEventDestroy(ev);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  std::vector<cudaStream_t> qs{c->side, c->side2};
  qs.insert(qs.end(), c->lane_st.begin(), c->lane_st.end());
  qs.insert(qs.end(), c->lane_side.begin(), c->lane_side.end());
  qs.insert(qs.end(), c->lane_side2.begin(), c->lane_side2.end());
  for (cudaStream_t q : qs)
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
  delete c;
}

// ------------------------------------------------------------ iteration
// lane l's view of the cache: the same cache fields, its own counters
static DevCache lane_cache(const mars_cache* c, int l) {
  DevCache d = c->dc;
  d.ctr = c->d_ctr + l;
  return d;
}

// lane l's share of the arena when nl lanes are in use: the l-th of nl equal
// slices of every slot array
static Arena lane_arena(const mars_cache* c, int l, int nl) {
  Arena a = c->arena;
  if (nl <= 1) return a;
  const uint64_t rc = c->arena.cap / (uint64_t)nl, sc = c->arena.scap / (uint64_t)nl;
  const uint64_t lc = c->arena.lcap / (uint64_t)nl, vc = c->arena.vcap / (uint64_t)nl;
  const uint64_t r0 = rc * (uint64_t)l, s0 = sc * (uint64_t)l, l0 = lc * (uint64_t)l, v0 = vc * (uint64_t)l;
  for (auto& p : a.R) p += r0;
  for (auto& p : a.V) p += r0;
  a.S += r0;
  a.M += r0;
  a.H += r0;
  for (auto& p : a.SH) p += s0;
  a.SL += s0;
  if (a.lcap) {
    a.R5 += r0;
    for (auto& p : a.LJ) p += l0;
    a.LR += l0;
    for (auto& p : a.LV) p += v0;
    a.LC += v0;
  }
  a.cap = rc;
  a.scap = sc;
  a.lcap = lc;
  a.vcap = vc;
  return a;
}

static mars_status poison(mars_cache* c, cudaError_t e, const char* what) {
  c->poisoned = true;
  return set_error(MARS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

mars_status render_iteration_impl(mars_cache* c, const mars_iter_params* p, float* image, mars_iter_stats* out,
                                  cudaStream_t st) {
  NvtxRange nvtx("mars:render_iteration");
  if (!c || !p) return set_error(MARS_ERR_INVALID_ARG, "null cache or params");
  if (c->poisoned) return set_error(MARS_ERR_CUDA, "cache is poisoned by an earlier CUDA error");
  if (p->iteration >= 65536u) return set_error(MARS_ERR_INVALID_ARG, "iteration %u >= 65536", p->iteration);
  if (p->mode < 0 || p->mode > 2) return set_error(MARS_ERR_INVALID_ARG, "bad mode %d", p->mode);
  if (p->mode == MARS_MODE_MARS && !c->has_estimate)
    return set_error(MARS_ERR_INVALID_ARG, "MARS mode needs a pixel estimate (run an iteration with update_estimate)");
  if (!(p->clamp_lo >= 0.0f) || !(p->clamp_hi <= 30.0f) || !(p->clamp_lo <= p->clamp_hi))
    return set_error(MARS_ERR_INVALID_ARG, "clamp range [%g, %g] outside [0, 30]", p->clamp_lo, p->clamp_hi);
  if (!(p->outlier > 0.0f)) return set_error(MARS_ERR_INVALID_ARG, "outlier multiple must be positive");
  if (!(p->max_multiplicity >= 0.0f)) return set_error(MARS_ERR_INVALID_ARG, "max_multiplicity must be >= 0");
  if (p->image_on_host && !image) return set_error(MARS_ERR_INVALID_ARG, "image_on_host without an image");
  if (p->vi_drop_brightest < 0 || p->vi_drop_brightest > MARS_MAX_DROP_BRIGHTEST ||
      (int64_t)p->vi_drop_brightest >= c->pixels)
    return set_error(MARS_ERR_INVALID_ARG, "vi_drop_brightest %d outside 0..%d (and below the pixel count)",
                     p->vi_drop_brightest, MARS_MAX_DROP_BRIGHTEST);
  if (p->combine < 0 || p->combine > 2) return set_error(MARS_ERR_INVALID_ARG, "combine %d outside 0..2", p->combine);
  if (p->combine && !p->update_estimate)
    return set_error(MARS_ERR_INVALID_ARG, "combine needs update_estimate (the weight is 1 / V_I)");
  // the pixel range of a shard (both 0: the whole frame)
  const bool ranged = p->px_begin != 0 || p->px_end != 0;
  if (ranged) {
    if (p->px_begin < 0 || (int64_t)p->px_end > c->pixels || p->px_begin >= p->px_end)
      return set_error(MARS_ERR_INVALID_ARG, "pixel range [%d, %d) outside [0, %lld)", p->px_begin, p->px_end,
                       (long long)c->pixels);
    if (p->update_estimate || p->combine)
      return set_error(MARS_ERR_INVALID_ARG, "a pixel range renders without update_estimate and combine (the "
                                             "image statistics need the whole frame)");
  }
  DeviceGuard g(c->device);
  if (!g.ok) return set_error(MARS_ERR_CUDA, "cannot select device %d", c->device);
  c->last_stream = st;
  if (inject_hit(g_inject_launch)) return poison(c, cudaErrorLaunchFailure, "injected render failure");
  const mars_scene* s = c->scene;

  IterArgs it{};
  it.seed = p->seed;
  it.job = p->job;
  it.iteration = p->iteration;
  it.mode = p->mode;
  it.aware = p->weights == MARS_WEIGHTS_AWARE;
  it.collect = p->collect != 0;
  it.has_estimate = c->has_estimate ? 1 : 0;
  it.clamp_lo = p->clamp_lo;
  it.clamp_hi = p->clamp_hi;
  it.outlier = p->outlier;
  it.max_mult = p->max_multiplicity;
  it.n_prev = c->n_iterations;
  it.drop_k = p->vi_drop_brightest;
  it.combine = p->combine;

  // reset the iteration counters (rays, vertices, beta sums, image sums)
  cudaError_t e = cudaMemsetAsync(c->d_ctr, 0, sizeof(DevCounters) * mars_cache::kMaxLanes, st);
  if (e != cudaSuccess) return poison(c, e, "counter reset");

  const int64_t npx = c->pixels;
  const int64_t r0 = ranged ? p->px_begin : 0, r1 = ranged ? p->px_end : npx, nr = r1 - r0;
  int ntiles = c->next_tiles > 0 ? c->next_tiles : 1;
  if (ntiles > c->max_tiles) ntiles = c->max_tiles;
  // Two lanes when each half of the image is expected to fit half of the
  // arena (the last iteration's use with the planner's headroom), the image is
  // large enough for two tiles to keep the GPU busy, and the iteration is not
  // profiled (a profiled iteration times each kernel alone on full-size
  // waves).  Otherwise one lane with the whole arena per tile.
  int iter_lanes = 1;
  if (c->use_lanes > 1 && !p->profile && nr >= c->lane_min_pixels && ntiles == 1 && 1.3 * c->last_need <= 1.0) {
    iter_lanes = (int)std::min<int64_t>(c->use_lanes, nr / std::max<int64_t>(1, c->lane_min_pixels / 2));
    ntiles = iter_lanes;
  }
  std::vector<std::pair<int64_t, int64_t>> tiles;
  for (int t = 0; t < ntiles; ++t) {
    const int64_t a = r0 + nr * t / ntiles, b = r0 + nr * (t + 1) / ntiles;
    if (b > a) tiles.emplace_back(a, b);
  }
  uint32_t retries = 0, used = 0, launches = 0, wave_launches = 0;
  uint64_t demand = 0;
  double trace_ms = 0.0, shade_ms = 0.0, shadow_ms = 0.0, reverse_ms = 0.0, image_ms = 0.0, light_ms = 0.0;
  float wave_ms[WAVE_KERNELS][MAXD] = {};
  const int D = c->max_depth;
  const int per_tile = 7 * D + 2;
  // A host image in page-locked memory is written by the image pass itself,
  // through its device address (no copy); any other host image is packed by
  // the image pass into a staging buffer of the cache (allocated on first use)
  // and read back in one copy.
  float* dev_out = image;
  bool staged = false;
  if (p->image_on_host) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, image) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
      dev_out = static_cast<float*>(pa.devicePointer);
    } else {
      cudaGetLastError();  // an unregistered pointer is not an error here
      staged = true;
      if (!c->d_host_stage &&
          (e = dev_alloc((void**)&c->d_host_stage, sizeof(float) * 3 * (size_t)npx, st)) != cudaSuccess)
        return set_error(e == cudaErrorMemoryAllocation ? MARS_ERR_OOM : MARS_ERR_CUDA, "staging alloc: %s",
                         cudaGetErrorString(e));
      dev_out = c->d_host_stage;
    }
  }
  while (true) {
    if (p->profile) {
      const size_t need = tiles.size() * per_tile + 2;
      while (c->events.size() < need) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return poison(c, e, "event create");
        c->events.push_back(ev);
      }
    }
    // the tiles' arguments: one pinned and one device slot per tile, copied
    // ahead of the launches that read them (the previous attempt has finished)
    for (size_t t = 0; t < tiles.size(); ++t) {
      IterArgs& a = c->h_args[t];
      a = it;
      a.tile_begin = (int)tiles[t].first;
      a.tile_end = (int)tiles[t].second;
      a.tile_slot = (int)t;
    }
    if ((e = cudaMemcpyAsync(c->d_args, c->h_args, sizeof(IterArgs) * tiles.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return poison(c, e, "argument copy");
    const bool profile = p->profile != 0;
    // Tiles go round-robin to the lanes; lane l has its own counters and its
    // 1/lanes share of the arena.  Lane 1 runs on its own streams, forked from
    // and joined to q, except in a profiled iteration, which times every
    // kernel alone on q.  Its totals are merged into lane 0's before the image
    // pass reads them.
    const int nl = std::min<int>(iter_lanes, (int)tiles.size());
    const bool concurrent = nl > 1 && !profile;
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
      cudaError_t r;
      if (concurrent) {
        if ((r = cudaEventRecord(c->fork_ev, q)) != cudaSuccess) return r;
        for (int l = 1; l < nl; ++l)
          if ((r = cudaStreamWaitEvent(c->lane_st[l - 1], c->fork_ev, 0)) != cudaSuccess) return r;
      }
      for (size_t t = 0; t < tiles.size(); ++t) {
        const int l = (int)(t % (size_t)nl);
        cudaEvent_t* ev = profile ? c->events.data() + t * per_tile : nullptr;
        const bool own = concurrent && l >= 1;
        cudaStream_t side2 = own ? (c->lane_side2.empty() ? nullptr : c->lane_side2[l - 1]) : c->side2;
        if ((r = launch_tile(s->ds, lane_cache(c, l), lane_arena(c, l, nl), c->d_args + t, c->launch,
                             own ? c->lane_st[l - 1] : q, own ? c->lane_side[l - 1] : c->side, side2,
                             own ? c->lane_sync[l - 1].data() : c->sync_events.data(), ev)) != cudaSuccess)
          return r;
      }
      if (nl > 1) {
        if (concurrent)
          for (int l = 1; l < nl; ++l)
            if ((r = cudaEventRecord(c->join_ev[l - 1], c->lane_st[l - 1])) != cudaSuccess ||
                (r = cudaStreamWaitEvent(q, c->join_ev[l - 1], 0)) != cudaSuccess)
              return r;
        for (int l = 1; l < nl; ++l)
          if ((r = launch_merge_lanes(c->d_ctr, c->d_ctr + l, q)) != cudaSuccess) return r;
      }
      cudaEvent_t* iev = profile ? c->events.data() + tiles.size() * per_tile : nullptr;
      if (iev) cudaEventRecord(iev[0], q);
      if (p->update_estimate) {
        if ((r = launch_image_stats(c->dc, s->width, s->height, c->d_args, dev_out, p->vi_drop_brightest > 0,
                                    p->combine != 0, c->scene->num_sms, q)) != cudaSuccess)
          return r;
      } else if (dev_out && ranged) {
        if ((r = launch_image_copy_range(c->dc, (int)r0, (int)r1, dev_out, q)) != cudaSuccess) return r;
      } else if (dev_out) {
        if ((r = launch_image_copy(c->dc, (int)npx, dev_out, q)) != cudaSuccess) return r;
      }
      if (iev) cudaEventRecord(iev[1], q);
      if ((r = cudaMemcpyAsync(c->h_tile_status, c->d_tile_status, sizeof(unsigned int) * tiles.size(),
                               cudaMemcpyDeviceToHost, q)) != cudaSuccess)
        return r;
      return cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, q);
    };
    // A first attempt with at most one tile per lane is replayed from a
    // recorded CUDA graph.  The legacy default stream cannot be captured, and a
    // profiled iteration times every launch with stream events: both launch
    // directly, as do the re-rendered tiles after an arena overflow.
    const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    if (c->use_graphs && capturable && !profile && retries == 0 && (int)tiles.size() <= iter_lanes) {
      GraphKey key;
      key.tiles = (int)tiles.size();
      key.update_estimate = p->update_estimate != 0;
      key.dev_out = dev_out;
      key.drop = p->vi_drop_brightest > 0;
      key.combine = p->combine != 0;
      key.r0 = ranged ? r0 : 0;
      key.r1 = ranged ? r1 : 0;
      key.L = c->launch;
      if (!c->graph_exec || !(c->graph_key == key)) {
        if (c->graph_exec) {
          cudaGraphExecDestroy(c->graph_exec);
          c->graph_exec = nullptr;
        }
        NvtxRange nvtx_capture("mars:graph_capture");
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
          return poison(c, e, "graph capture");
        const cudaError_t ee = enqueue(st);
        e = cudaStreamEndCapture(st, &graph);
        if (ee != cudaSuccess || e != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return poison(c, ee != cudaSuccess ? ee : e, "graph capture");
        }
        e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          c->graph_exec = nullptr;
          return poison(c, e, "graph instantiate");
        }
        c->graph_key = key;
        c->graph_captures += 1;
      }
      if ((e = cudaGraphLaunch(c->graph_exec, st)) != cudaSuccess) return poison(c, e, "graph launch");
    } else if ((e = enqueue(st)) != cudaSuccess) {
      return poison(c, e, "render launch");
    }
    launches += (uint32_t)(tiles.size() * tile_launches(D, c->techniques)) + (uint32_t)(nl - 1);
    wave_launches += (uint32_t)(tiles.size() * D);
    launches += p->update_estimate ? 3 + (p->vi_drop_brightest > 0 ? 2 : 0) + (p->combine ? 1 : 0)
                                   : (dev_out ? 1 : 0);
    used += (uint32_t)tiles.size();
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return poison(c, e, "render");
    if (p->profile) {
      for (size_t t = 0; t < tiles.size(); ++t) {
        cudaEvent_t* ev = c->events.data() + t * per_tile;
        float ms = 0.f;
        // event layout: see launch_tile
        for (int d = 1; d <= D; ++d) {
          cudaEventElapsedTime(&ms, ev[2 * (d - 1)], ev[2 * (d - 1) + 1]);
          trace_ms += ms;
          wave_ms[WK_TRACE][d - 1] += ms;
          cudaEventElapsedTime(&ms, ev[2 * (d - 1) + 1], ev[2 * (d - 1) + 2]);
          shade_ms += ms;
          wave_ms[WK_SHADE][d - 1] += ms;
          if (d <= D - 1 && (c->techniques & MARS_TECH_NEE)) {
            cudaEventElapsedTime(&ms, ev[2 * D + 2 * (d - 1) + 1], ev[2 * D + 2 * (d - 1) + 2]);
            shadow_ms += ms;
            wave_ms[WK_SHADOW][d - 1] += ms;
          }
          if (d <= D - 2 && (c->techniques & MARS_TECH_LIGHT)) {
            cudaEventElapsedTime(&ms, ev[5 * D + 2 + 2 * (d - 1)], ev[5 * D + 2 + 2 * (d - 1) + 1]);
            light_ms += ms;
          }
        }
        // the k-th reverse launch (k = 1..D) handles wave D - k + 1
        for (int k = 1; k <= D; ++k) {
          cudaEventElapsedTime(&ms, k == 1 ? ev[5 * D + 1] : ev[4 * D + k - 1], ev[4 * D + k]);
          reverse_ms += ms;
          wave_ms[WK_REVERSE][D - k] += ms;
        }
      }
      float ms = 0.f;
      cudaEvent_t* iev = c->events.data() + tiles.size() * per_tile;
      cudaEventElapsedTime(&ms, iev[0], iev[1]);
      image_ms += ms;
    }
    demand = std::max<uint64_t>(demand, c->h_ctr->demand);
    // Each overflowed tile is split into k pieces.  k comes from the last tile
    // of the attempt: it had filled `demand` slots when its first dstar waves
    // were allocated; with the remaining waves taken as large as those, it
    // needed about demand x D / dstar slots (at least a halving, at most 16).
    int k = 2;
    {
      const DevCounters& hc = *c->h_ctr;
      int dstar = 1;
      for (int d = 1; d <= D; ++d)
        if (hc.count[d] > 0) dstar = d;
      const double est = (double)hc.demand * (double)D / (double)dstar;
      const double tcap = (double)(c->arena.cap / (uint64_t)std::max(1, nl));
      k = std::min(16, std::max(2, (int)std::ceil(1.3 * est / tcap)));
    }
    std::vector<std::pair<int64_t, int64_t>> again;
    for (size_t t = 0; t < tiles.size(); ++t) {
      if (!c->h_tile_status[t]) continue;
      const int64_t a = tiles[t].first, b = tiles[t].second;
      if (b - a <= 1)
        return set_error(MARS_ERR_OOM, "one pixel's path tree needs more than the arena's %llu rays",
                         (unsigned long long)(c->arena.cap / (uint64_t)std::max(1, nl)));
      const int64_t parts = std::min<int64_t>(k, b - a);
      for (int64_t j = 0; j < parts; ++j) again.emplace_back(a + (b - a) * j / parts, a + (b - a) * (j + 1) / parts);
    }
    if (again.empty()) break;
    if ((int)again.size() > c->max_tiles) return set_error(MARS_ERR_OOM, "too many tiles after arena overflow");
    retries += (uint32_t)again.size();
    tiles.swap(again);
    // the committed tiles stay; clear the overflow marker so the image pass runs
    if ((e = cudaMemsetAsync(&c->d_ctr->any_overflow, 0, sizeof(unsigned int), st)) != cudaSuccess)
      return poison(c, e, "overflow reset");
  }
  // plan the next iteration's tiles from this one's committed arena use: a
  // tile holds every depth wave of its pixels, about entries x (tile pixels /
  // pixels) ray slots (and shadow slots likewise); 30 % headroom for the uneven
  // spread of path trees over the image, times the growth over the previous
  // iteration (up to 2x: the learned counts ramp up over the first MARS
  // iterations); a tile that still overflows is split and re-rendered as above
  {
    const DevCounters& h = *c->h_ctr;
    double need = std::max((double)h.entries / (double)c->arena.cap,
                           (double)h.shadow_entries / (double)c->arena.scap);
    if (c->arena.lcap) need = std::max(need, (double)h.light_entries / (double)c->arena.lcap);
    if (c->arena.vcap) need = std::max(need, (double)h.light_vertex_entries / (double)c->arena.vcap);
    const double growth = c->last_entries > 0 ? std::min(2.0, std::max(1.0, (double)h.entries /
                                                                             (double)c->last_entries))
                                              : 1.0;
    const int t = (int)std::ceil(need * 1.3 * growth);
    c->next_tiles = std::min(c->max_tiles, std::max(1, t));
    c->last_entries = h.entries;
    c->last_need = need;
  }
  if (p->update_estimate) {
    c->n_iterations += 1;
    c->has_estimate = true;
  }
  if (staged) {
    if ((e = cudaMemcpyAsync(image + 3 * (size_t)r0, c->d_host_stage + 3 * (size_t)r0, sizeof(float) * 3 * (size_t)nr,
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return poison(c, e, "image copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return poison(c, e, "image copy");
  }
  if (out) {
    const DevCounters& h = *c->h_ctr;
    out->VI = h.VI;
    out->CI = h.CI;
    out->rays = h.rays;
    out->vertices = h.vertices + h.light_rays;  // closest-hit queries of camera and light paths
    out->estimator_vertices = h.est_vertices;
    for (int t = 0; t < NT; ++t) out->mean_beta[t] = h.est_vertices ? h.sum_beta[t] / (double)h.est_vertices : 0.0;
    out->tiles = used;
    out->retries = retries;
    out->arena_demand = demand;
    out->launches = launches;
    out->wave_launches = wave_launches;
    out->trace_ms = trace_ms;
    out->shade_ms = shade_ms;
    out->shadow_ms = shadow_ms;
    out->reverse_ms = reverse_ms;
    out->image_ms = image_ms;
    out->wave_entries = h.entries;
    out->shadow_entries = h.shadow_entries;
    out->shadow_traced = h.shadow_traced;
    for (int k = 0; k < WAVE_KERNELS; ++k)
      for (int d = 0; d < MAXD; ++d) out->wave_ms[k][d] = wave_ms[k][d];
    for (int d = 0; d < MAXD; ++d) out->wave_rays[d] = h.wave_total[d + 1];
    for (int k = 0; k < 2; ++k)
      for (int q = 0; q < 4; ++q) out->trace_work[k][q] = h.trace_work[k][q];
    out->check_flags = h.check_flags;
    out->reserved = 0;
    out->light_rays = h.light_rays;
    out->connection_rays = h.conn_rays;
    out->light_samples = h.light_entries;
    out->light_ms = light_ms;
  }
  return MARS_OK;
}

mars_status update_counts_impl(mars_cache* c, cudaStream_t st) {
  NvtxRange nvtx("mars:update_counts");
  if (!c) return set_error(MARS_ERR_INVALID_ARG, "null cache");
  if (c->poisoned) return set_error(MARS_ERR_CUDA, "cache is poisoned by an earlier CUDA error");
  DeviceGuard g(c->device);
  if (inject_hit(g_inject_launch)) return poison(c, cudaErrorLaunchFailure, "injected update failure");
  c->last_stream = st;
  cudaError_t e = cudaSuccess;
  if (c->dc.oct_nodes && (e = launch_leaf_samples(c->dc, st)) != cudaSuccess) return poison(c, e, "update launch");
  if ((e = launch_update(c->dc, c->scene->num_sms, st)) != cudaSuccess) return poison(c, e, "update launch");
  if (c->dc.oct_nodes && (e = launch_octree_refine(c->dc, c->scene->num_sms, st)) != cudaSuccess)
    return poison(c, e, "octree refine launch");
  // the next training iteration averages its own V_I and C_I
  if ((e = cudaMemsetAsync(c->d_img_acc, 0, 3 * sizeof(double), st)) != cudaSuccess)
    return poison(c, e, "image statistics reset");
  return MARS_OK;
}

mars_status get_state_impl(mars_cache* c, mars_cache_state* s, cudaStream_t st) {
  if (!c || !s) return set_error(MARS_ERR_INVALID_ARG, "null cache or state");
  if (c->poisoned) return set_error(MARS_ERR_CUDA, "cache is poisoned by an earlier CUDA error");
  DeviceGuard g(c->device);
  if (c->dc.oct_nodes) {
    int meta[3] = {0, 0, 0};
    cudaError_t e0;
    if ((e0 = cudaMemcpyAsync(meta, c->d_oct_meta, sizeof(int) * 3, cudaMemcpyDeviceToHost, st)) ||
        (e0 = cudaStreamSynchronize(st)))
      return poison(c, e0, "state copy");
    s->oct_n_nodes = meta[0];
    s->oct_n_leaves = meta[1];
    if ((s->oct_nodes && (e0 = cudaMemcpyAsync(s->oct_nodes, c->d_oct_nodes, sizeof(int) * meta[0],
                                                cudaMemcpyDeviceToHost, st))) ||
        (s->oct_leaf_level && (e0 = cudaMemcpyAsync(s->oct_leaf_level, c->d_oct_level, sizeof(int) * meta[1],
                                                     cudaMemcpyDeviceToHost, st))))
      return poison(c, e0, "state copy");
  } else {
    s->oct_n_nodes = s->oct_n_leaves = 0;
  }
  const int64_t cells = c->cells, px = c->pixels;
  const bool guided = c->techniques & MARS_TECH_GUIDED;
  cudaError_t e = cudaSuccess;
  std::vector<float4> cnt;
  std::vector<float4> img4;
  if (s->q_rr || s->q_s || s->valid) {
    cnt.resize(2 * NT * cells);
    e = cudaMemcpyAsync(cnt.data(), c->d_cnt, sizeof(float4) * cnt.size(), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return poison(c, e, "state copy");
  }
  std::vector<float> s32;
  std::vector<double> s64;
  if (s->stats && c->fp32_stats) {
    s32.resize((size_t)NSTAT * NT * cells);
    if ((e = cudaMemcpyAsync(s32.data(), c->d_stats32, sizeof(float) * s32.size(), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return poison(c, e, "state copy");
  } else if (s->stats) {
    // device layout: structure of arrays [stat][cell][technique]
    s64.resize((size_t)NSTAT * NT * cells);
    if ((e = cudaMemcpyAsync(s64.data(), c->d_stats, sizeof(double) * s64.size(), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return poison(c, e, "state copy");
  }
  if (s->guide_hist && guided &&
      (e = cudaMemcpyAsync(s->guide_hist, c->d_hist, sizeof(float) * GUIDE_BINS * cells, cudaMemcpyDeviceToHost,
                           st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if (s->guide_cdf && guided &&
      (e = cudaMemcpyAsync(s->guide_cdf, c->d_cdf, sizeof(float) * GUIDE_BINS * cells, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
    return poison(c, e, "state copy");
  if (s->pixel_estimate &&
      (e = cudaMemcpy2DAsync(s->pixel_estimate, 3 * sizeof(float), c->d_est, sizeof(float4), 3 * sizeof(float),
                             (size_t)px, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if (s->run_sum &&
      (e = cudaMemcpy2DAsync(s->run_sum, 3 * sizeof(float), c->d_run, sizeof(float4), 3 * sizeof(float), (size_t)px,
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  // the fourth channel of the iteration image holds each pixel's ray count
  if (s->pixel_rays &&
      (e = cudaMemcpy2DAsync(s->pixel_rays, sizeof(float), reinterpret_cast<const float*>(c->d_img) + 3,
                             sizeof(float4), sizeof(float), (size_t)px, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return poison(c, e, "state copy");
  for (size_t k = 0; k < s32.size(); ++k) s->stats[k] = (double)s32[k];
  if (!s64.empty()) {
    const size_t plane = (size_t)NT * cells;
    for (size_t k = 0; k < plane; ++k)
      for (int q = 0; q < NSTAT; ++q) s->stats[k * NSTAT + q] = s64[q * plane + k];
  }
  for (int64_t k = 0; k < cells * NT && !cnt.empty(); ++k) {
    const float4 r = cnt[2 * k], q = cnt[2 * k + 1];
    if (s->q_rr) { s->q_rr[3 * k] = r.x; s->q_rr[3 * k + 1] = r.y; s->q_rr[3 * k + 2] = r.z; }
    if (s->q_s) { s->q_s[3 * k] = q.x; s->q_s[3 * k + 1] = q.y; s->q_s[3 * k + 2] = q.z; }
    if (s->valid) s->valid[k] = r.w > 0.0f ? 1 : 0;
  }
  s->n_iterations = c->n_iterations;
  s->has_estimate = c->has_estimate ? 1 : 0;
  double acc[3] = {0.0, 0.0, 0.0};
  if ((e = cudaMemcpyAsync(acc, c->d_img_acc, sizeof(acc), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return poison(c, e, "state copy");
  s->image_iterations = (int32_t)acc[2];
  s->VI = acc[2] > 0.0 ? acc[0] / acc[2] : 0.0;
  s->CI = acc[2] > 0.0 ? acc[1] / acc[2] : 0.0;
  return MARS_OK;
}

mars_status set_state_impl(mars_cache* c, const mars_cache_state* s, cudaStream_t st) {
  if (!c || !s) return set_error(MARS_ERR_INVALID_ARG, "null cache or state");
  if (c->poisoned) return set_error(MARS_ERR_CUDA, "cache is poisoned by an earlier CUDA error");
  if (s->n_iterations < 0) return set_error(MARS_ERR_INVALID_ARG, "negative n_iterations");
  DeviceGuard g(c->device);
  const int64_t cells = c->cells, px = c->pixels;
  const bool guided = c->techniques & MARS_TECH_GUIDED;
  cudaError_t e = cudaSuccess;
  if (s->oct_nodes) {
    if (!c->dc.oct_nodes) return set_error(MARS_ERR_INVALID_ARG, "octree state for a grid cache");
    const int nn = s->oct_n_nodes, nl = s->oct_n_leaves;
    if (nn < 1 || nn > c->oct_cap_nodes || nl < 1 || nl > cells || !s->oct_leaf_level)
      return set_error(MARS_ERR_INVALID_ARG, "octree state: %d nodes, %d leaves out of range", nn, nl);
    // check the tree before any kernel descends it: every node reached once
    // from the root within the level limit, internal nodes' 8 children in
    // range, every leaf cell in range exactly once, levels as given
    std::vector<int> lnode((size_t)cells, -1), depth((size_t)nn, -1);
    std::vector<std::pair<int, int>> stack{{0, 0}};
    int leaves = 0;
    bool ok = true;
    while (!stack.empty() && ok) {
      const auto [k, lev] = stack.back();
      stack.pop_back();
      if (depth[k] >= 0) { ok = false; break; }
      depth[k] = lev;
      const int v = s->oct_nodes[k];
      if (v < 0) {
        const int cell = ~v;
        if (cell >= nl || lnode[cell] >= 0 || s->oct_leaf_level[cell] != lev) { ok = false; break; }
        lnode[cell] = k;
        ++leaves;
      } else {
        if (lev >= OCT_LMAX || v < 1 || v + 7 >= nn) { ok = false; break; }
        for (int o = 0; o < 8; ++o) stack.push_back({v + o, lev + 1});
      }
    }
    if (!ok || leaves != nl) return set_error(MARS_ERR_INVALID_ARG, "octree state: not a valid tree");
    const int meta[3] = {nn, nl, 0};
    for (auto& x : lnode) x = x < 0 ? 0 : x;
    if ((e = cudaMemcpyAsync(c->d_oct_nodes, s->oct_nodes, sizeof(int) * nn, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_oct_level, s->oct_leaf_level, sizeof(int) * nl, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_oct_lnode, lnode.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(c->d_oct_meta, meta, sizeof(int) * 3, cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st)))
      return poison(c, e, "state copy");
  }
  if (s->q_rr || s->q_s || s->valid) {
    std::vector<float4> cnt(2 * NT * cells);
    if ((e = cudaMemcpy(cnt.data(), c->d_cnt, sizeof(float4) * cnt.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return poison(c, e, "state copy");
    for (int64_t k = 0; k < cells * NT; ++k) {
      float4& r = cnt[2 * k];
      float4& q = cnt[2 * k + 1];
      if (s->q_rr) { r.x = s->q_rr[3 * k]; r.y = s->q_rr[3 * k + 1]; r.z = s->q_rr[3 * k + 2]; }
      if (s->q_s) { q.x = s->q_s[3 * k]; q.y = s->q_s[3 * k + 1]; q.z = s->q_s[3 * k + 2]; }
      if (s->valid) r.w = s->valid[k] ? 1.0f : 0.0f;
    }
    if ((e = cudaMemcpyAsync(c->d_cnt, cnt.data(), sizeof(float4) * cnt.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return poison(c, e, "state copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return poison(c, e, "state copy");
  }
  std::vector<double> s64;
  std::vector<float> s32;
  if (s->stats && c->fp32_stats) {
    s32.resize((size_t)NSTAT * NT * cells);
    for (size_t k = 0; k < s32.size(); ++k) s32[k] = (float)s->stats[k];
    if ((e = cudaMemcpyAsync(c->d_stats32, s32.data(), sizeof(float) * s32.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return poison(c, e, "state copy");
  } else if (s->stats) {
    const size_t plane = (size_t)NT * cells;
    s64.resize((size_t)NSTAT * plane);
    for (size_t k = 0; k < plane; ++k)
      for (int q = 0; q < NSTAT; ++q) s64[q * plane + k] = s->stats[k * NSTAT + q];
    if ((e = cudaMemcpyAsync(c->d_stats, s64.data(), sizeof(double) * s64.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return poison(c, e, "state copy");
  }
  if (s->guide_hist && guided &&
      (e = cudaMemcpyAsync(c->d_hist, s->guide_hist, sizeof(float) * GUIDE_BINS * cells, cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if (s->guide_cdf && guided &&
      (e = cudaMemcpyAsync(c->d_cdf, s->guide_cdf, sizeof(float) * GUIDE_BINS * cells, cudaMemcpyHostToDevice, st)) !=
          cudaSuccess)
    return poison(c, e, "state copy");
  // a histogram or CDF from outside: the next update rebuilds every cell's CDF
  if ((s->guide_hist || s->guide_cdf) && guided &&
      (e = cudaMemsetAsync(c->d_guide_dirty, 1, (size_t)cells, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if (s->pixel_estimate &&
      (e = cudaMemcpy2DAsync(c->d_est, sizeof(float4), s->pixel_estimate, 3 * sizeof(float), 3 * sizeof(float),
                             (size_t)px, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if (s->run_sum &&
      (e = cudaMemcpy2DAsync(c->d_run, sizeof(float4), s->run_sum, 3 * sizeof(float), 3 * sizeof(float), (size_t)px,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  // V_I and C_I feed the next update: the means of image_iterations iterations
  // (one when it is 0 and either is set)
  const int32_t ni = s->image_iterations > 0 ? s->image_iterations : (s->VI != 0.0 || s->CI != 0.0 ? 1 : 0);
  const double acc[3] = {s->VI * ni, s->CI * ni, (double)ni};
  if ((e = cudaMemcpyAsync(c->d_img_acc, acc, sizeof(acc), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return poison(c, e, "state copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return poison(c, e, "state copy");
  c->n_iterations = s->n_iterations;
  c->has_estimate = s->has_estimate != 0;
  return MARS_OK;
}

}  // namespace mars

// ======================================================================= C ABI
using namespace mars;

extern "C" {

mars_status mars_scene_create(const mars_scene_desc* desc, void* stream, mars_scene** out) {
  return scene_create_impl(desc, (cudaStream_t)stream, out);
}

mars_status mars_scene_destroy(mars_scene* scene) {
  scene_destroy_impl(scene);
  return MARS_OK;
}

mars_status mars_cache_create(const mars_scene* scene, const mars_cache_desc* desc, void* stream, mars_cache** out) {
  return cache_create_impl(scene, desc, (cudaStream_t)stream, out);
}

mars_status mars_cache_destroy(mars_cache* cache) {
  cache_destroy_impl(cache);
  return MARS_OK;
}

mars_status mars_cache_info_get(const mars_cache* c, mars_cache_info* info) {
  if (!c || !info) return set_error(MARS_ERR_INVALID_ARG, "null cache or info");
  info->n_cells = c->cells;
  info->n_pixels = c->pixels;
  info->grid_n = c->grid_n;
  info->techniques = c->techniques;
  info->max_depth = c->max_depth;
  info->n_prims = c->scene->n_prims;
  info->arena_capacity = c->arena.cap;
  info->device_bytes = c->device_bytes + c->scene->device_bytes;
  info->device = c->device;
  info->n_lights = c->scene->n_lights;
  info->oct_cap_nodes = c->oct_cap_nodes;
  info->oct_n_nodes = info->oct_n_leaves = 0;
  info->graph_captures = c->graph_captures;
  if (c->dc.oct_nodes) {
    DeviceGuard g(c->device);
    int meta[3] = {0, 0, 0};
    if (cudaMemcpy(meta, c->d_oct_meta, sizeof(int) * 3, cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_error(MARS_ERR_CUDA, "octree size read failed");
    info->oct_n_nodes = meta[0];
    info->oct_n_leaves = meta[1];
  }
  return MARS_OK;
}

mars_status mars_render_iteration(mars_cache* cache, const mars_iter_params* params, float* image_rgb,
                                  mars_iter_stats* stats_host, void* stream) {
  return render_iteration_impl(cache, params, image_rgb, stats_host, (cudaStream_t)stream);
}

mars_status mars_update_counts(mars_cache* cache, void* stream) {
  return update_counts_impl(cache, (cudaStream_t)stream);
}

mars_status mars_cache_get_state(mars_cache* cache, mars_cache_state* state, void* stream) {
  return get_state_impl(cache, state, (cudaStream_t)stream);
}

mars_status mars_debug_inject_failure(int32_t kind, int32_t n) {
  if (n < 0) return set_error(MARS_ERR_INVALID_ARG, "negative countdown %d", n);
  if (kind == MARS_INJECT_ALLOC)
    g_inject_alloc.store(n);
  else if (kind == MARS_INJECT_LAUNCH)
    g_inject_launch.store(n);
  else
    return set_error(MARS_ERR_INVALID_ARG, "unknown injection kind %d", kind);
  return MARS_OK;
}

mars_status mars_cache_combined_image(mars_cache* c, float* image_rgb, double* weight_sum, void* stream) {
  if (!c) return set_error(MARS_ERR_INVALID_ARG, "null cache");
  if (c->poisoned) return set_error(MARS_ERR_CUDA, "cache is poisoned by an earlier CUDA error");
  DeviceGuard g(c->device);
  if (!g.ok) return set_error(MARS_ERR_CUDA, "cannot select device %d", c->device);
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  const int64_t npx = c->pixels;
  cudaError_t e;
  if (image_rgb) {
    if (!c->d_host_stage &&
        (e = dev_alloc((void**)&c->d_host_stage, sizeof(float) * 3 * (size_t)npx, st)) != cudaSuccess)
      return set_error(e == cudaErrorMemoryAllocation ? MARS_ERR_OOM : MARS_ERR_CUDA, "staging alloc: %s",
                       cudaGetErrorString(e));
    if ((e = launch_combined_out(c->dc, (int)npx, c->d_host_stage, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(image_rgb, c->d_host_stage, sizeof(float) * 3 * (size_t)npx, cudaMemcpyDeviceToHost,
                             st)) != cudaSuccess)
      return poison(c, e, "combined image");
  }
  double w = 0.0;
  if ((e = cudaMemcpyAsync(&w, c->d_comb_w, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return poison(c, e, "combined image");
  if (weight_sum) *weight_sum = w;
  return MARS_OK;
}

mars_status mars_cache_set_state(mars_cache* cache, const mars_cache_state* state, void* stream) {
  return set_state_impl(cache, state, (cudaStream_t)stream);
}

mars_status mars_cache_get_launch(const mars_cache* c, mars_launch_config* out) {
  if (!c || !out) return set_error(MARS_ERR_INVALID_ARG, "null cache or output");
  for (int k = 0; k < WAVE_KERNELS; ++k) {
    out->threads[k] = c->launch.threads[k];
    out->blocks_per_sm[k] = c->blocks_per_sm[k];
    out->max_registers[k] = wave_variant_registers(k, c->launch.variant[k]);
  }
  out->lanes = c->use_lanes;
  out->lane_min_pixels = (int32_t)std::min<int64_t>(c->lane_min_pixels, INT32_MAX);
  return MARS_OK;
}

static bool variant_of(int kernel, int regs, int* v) {
  for (int k = 0; k < wave_variants(kernel); ++k)
    if (wave_variant_registers(kernel, k) == regs) {
      *v = k;
      return true;
    }
  return false;
}

mars_status mars_cache_set_launch(mars_cache* c, const mars_launch_config* cfg) {
  if (!c || !cfg) return set_error(MARS_ERR_INVALID_ARG, "null cache or config");
  int var[WAVE_KERNELS];
  for (int k = 0; k < WAVE_KERNELS; ++k)
    if (!variant_of(k, cfg->max_registers[k], &var[k]))
      return set_error(MARS_ERR_INVALID_ARG, "wave kernel %d: no variant capped at %d registers", k,
                       cfg->max_registers[k]);
  if (cfg->lanes < 0 || cfg->lanes > c->lanes)
    return set_error(MARS_ERR_INVALID_ARG, "lanes %d outside 1..%d (the cache's lanes)", cfg->lanes, c->lanes);
  if (cfg->lane_min_pixels < 0 || cfg->lane_min_pixels == 1)
    return set_error(MARS_ERR_INVALID_ARG, "lane_min_pixels %d below 2", cfg->lane_min_pixels);
  DeviceGuard g(c->device);
  const mars_status rc = apply_launch(c, cfg->threads, cfg->blocks_per_sm, var);
  if (rc != MARS_OK) return rc;
  if (cfg->lanes > 0) c->use_lanes = cfg->lanes;
  if (cfg->lane_min_pixels > 0) c->lane_min_pixels = cfg->lane_min_pixels;
  return MARS_OK;
}

// Coordinate search over the launch shape of each wave kernel in turn (register
// cap variant x threads per block x blocks per SM), timing the kernel's own
// CUDA events over `repeats` renders of the given iteration without
// statistics, image statistics or guide deposits, so the cache's state is left
// as it was.
mars_status mars_cache_autotune(mars_cache* c, const mars_iter_params* params, int32_t repeats,
                                mars_launch_config* chosen, void* stream) {
  NvtxRange nvtx("mars:autotune");
  if (!c || !params) return set_error(MARS_ERR_INVALID_ARG, "null cache or params");
  if (repeats < 1 || repeats > 100) return set_error(MARS_ERR_INVALID_ARG, "repeats %d outside 1..100", repeats);
  if (c->poisoned) return set_error(MARS_ERR_CUDA, "cache is poisoned by an earlier CUDA error");
  DeviceGuard g(c->device);
  mars_iter_params p = *params;
  p.collect = 0;
  p.update_estimate = 0;
  p.image_on_host = 0;
  p.combine = 0;
  p.profile = 1;
  int threads[WAVE_KERNELS], bps[WAVE_KERNELS], var[WAVE_KERNELS];
  for (int k = 0; k < WAVE_KERNELS; ++k) {
    threads[k] = c->launch.threads[k];
    bps[k] = c->blocks_per_sm[k];
    var[k] = c->launch.variant[k];
  }
  auto time_of = [&](int k, double* ms) -> mars_status {
    mars_status rc = apply_launch(c, threads, bps, var);
    if (rc != MARS_OK) return rc;
    double tot = 0.0;
    for (int r = 0; r <= repeats; ++r) {  // the first render warms up
      mars_iter_stats st{};
      rc = render_iteration_impl(c, &p, nullptr, &st, (cudaStream_t)stream);
      if (rc != MARS_OK) return rc;
      const double v[WAVE_KERNELS] = {st.trace_ms, st.shade_ms, st.shadow_ms, st.reverse_ms};
      if (r > 0) tot += v[k];
    }
    *ms = tot / repeats;
    return MARS_OK;
  };
  const int cand_threads[3] = {64, 128, 256};
  for (int k = 0; k < WAVE_KERNELS; ++k) {
    if (k == WK_SHADOW && !(c->techniques & MARS_TECH_NEE)) continue;
    int best_t = threads[k], best_b = bps[k], best_v = var[k];
    double best = 1e300;
    for (int v = 0; v < wave_variants(k); ++v) {
      for (int ti = 0; ti < 3; ++ti) {
        int occ[WAVE_KERNELS];
        int tt[WAVE_KERNELS] = {threads[0], threads[1], threads[2], threads[3]};
        int vv[WAVE_KERNELS] = {var[0], var[1], var[2], var[3]};
        tt[k] = cand_threads[ti];
        vv[k] = v;
        if (wave_occupancy(tt, vv, occ) != cudaSuccess) return set_error(MARS_ERR_CUDA, "occupancy query failed");
        const int o = std::max(1, occ[k]);
        const int cand_b[3] = {std::max(1, o / 2), o, 2 * o};
        for (int bi = 0; bi < 3; ++bi) {
          if (bi == 0 && cand_b[0] == o) continue;
          threads[k] = cand_threads[ti];
          var[k] = v;
          bps[k] = std::min(64, cand_b[bi]);
          double ms = 0.0;
          const mars_status rc = time_of(k, &ms);
          if (rc != MARS_OK) return rc;
          if (ms < best) {
            best = ms;
            best_t = threads[k];
            best_b = bps[k];
            best_v = var[k];
          }
        }
      }
    }
    threads[k] = best_t;
    bps[k] = best_b;
    var[k] = best_v;
  }
  mars_status rc = apply_launch(c, threads, bps, var);
  if (rc != MARS_OK) return rc;
  // Tile lanes: whole iterations as rendered outside profiling (graph replay,
  // concurrent lanes), one lane against all of them, timed on the stream.
  if (c->lanes > 1 && c->pixels >= kLaneFloorPixels) {
    mars_iter_params q = p;
    q.profile = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return set_error(MARS_ERR_CUDA, "event create failed");
    }
    const int cand_lanes[2] = {1, c->lanes};
    const int64_t cand_min[2] = {c->lane_min_pixels,
                                 std::max<int64_t>(kLaneFloorPixels, std::min<int64_t>(kLaneMinPixels, c->pixels))};
    double best = 1e300;
    int best_k = 0;
    for (int k = 0; k < 2 && rc == MARS_OK; ++k) {
      c->use_lanes = cand_lanes[k];
      c->lane_min_pixels = cand_min[k];
      double tot = 0.0;
      for (int r = 0; r <= repeats && rc == MARS_OK; ++r) {  // the first render warms up (and records the graph)
        mars_iter_stats st{};
        float ms = 0.f;
        if (cudaEventRecord(e0, (cudaStream_t)stream) != cudaSuccess) rc = set_error(MARS_ERR_CUDA, "event record");
        if (rc == MARS_OK) rc = render_iteration_impl(c, &q, nullptr, &st, (cudaStream_t)stream);
        if (rc == MARS_OK && (cudaEventRecord(e1, (cudaStream_t)stream) != cudaSuccess ||
                              cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          rc = set_error(MARS_ERR_CUDA, "event timing");
        if (r > 0) tot += ms;
      }
      if (rc == MARS_OK && tot < best) {
        best = tot;
        best_k = k;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MARS_OK) return rc;
    c->use_lanes = cand_lanes[best_k];
    c->lane_min_pixels = cand_min[best_k];
  }
  if (chosen) return mars_cache_get_launch(c, chosen);
  return MARS_OK;
}

const char* mars_last_error_string(void) { return g_last_error.c_str(); }

const char* mars_version(void) { return "mars-gb300 0.1 (sm_103a)"; }

int32_t mars_training_step_ends(int32_t iteration, int32_t warmup, int32_t iterations) {
  if (iteration < 0 || iteration >= iterations || warmup < 0) return 0;
  if (iteration < warmup || iteration == iterations - 1) return 1;
  // after warm-up: training iterations of 1, 2, 4, ... renders end where the
  // renders so far, k + 1, are 2^m - 1, unless fewer renders than the ending
  // iteration's 2^(m-1) would remain (they join it)
  const int64_t k2 = (int64_t)(iteration - warmup) + 2;
  const int64_t left = (int64_t)iterations - 1 - iteration;
  return (k2 & (k2 - 1)) == 0 && left >= k2 / 2 ? 1 : 0;
}

}  // extern "C"
