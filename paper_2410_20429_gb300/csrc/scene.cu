// scene.cu -- linear BVH construction on the device (Karras, "Maximizing
// Parallelism in the Construction of BVHs, Octrees, and k-d Trees", HPG 2012):
// 30-bit Morton codes of the primitive centroids (above a size-class bit) with
// the primitive index as a tie-breaking low word, a bitonic sort, one thread per internal node to find
// its key range and split, and a bottom-up pass that fills the child bounds
// (the second thread to reach a node computes it).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace mars {

namespace {

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

// keys[i] = large << 62 | morton(centroid) << 32 | i ; padding keys are all ones.
// A primitive whose box spans at least half the scene's largest extent (a wall,
// a floor) is "large": the flag bit makes the hierarchy's first split separate
// the large primitives from the small ones, so no subtree of small primitives
// carries a box inflated by a wall.
__global__ void k_morton(const float4* __restrict__ box, int n, int npow, float lo0, float lo1, float lo2,
                         float ie0, float ie1, float ie2, float large_extent, unsigned long long* keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npow) return;
  if (i >= n) {
    keys[i] = ~0ull;
    return;
  }
  const float4 blo = box[2 * i], bhi = box[2 * i + 1];
  const float c[3] = {0.5f * (blo.x + bhi.x), 0.5f * (blo.y + bhi.y), 0.5f * (blo.z + bhi.z)};
  const float lo[3] = {lo0, lo1, lo2}, ie[3] = {ie0, ie1, ie2};
  uint32_t q[3];
  for (int a = 0; a < 3; ++a) {
    float f = (c[a] - lo[a]) * ie[a] * 1024.0f;
    f = fminf(fmaxf(f, 0.0f), 1023.0f);
    q[a] = (uint32_t)f;
  }
  const uint32_t m = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
  const float span = fmaxf(fmaxf(bhi.x - blo.x, bhi.y - blo.y), bhi.z - blo.z);
  const unsigned long long large = span >= large_extent ? 1ull : 0ull;
  keys[i] = (large << 62) | ((unsigned long long)m << 32) | (unsigned long long)i;
}

__global__ void k_bitonic(unsigned long long* keys, int npow, int j, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npow) return;
  const int l = i ^ j;
  if (l <= i) return;
  const unsigned long long a = keys[i], b = keys[l];
  const bool up = (i & k) == 0;
  if ((up && a > b) || (!up && a < b)) {
    keys[i] = b;
    keys[l] = a;
  }
}

__device__ __forceinline__ int delta(const unsigned long long* k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(k[i] ^ k[j]);
}

// internal node i of n-1: children encoded as internal index (>= 0) or ~leaf slot
__global__ void k_hierarchy(const unsigned long long* __restrict__ keys, int n, int2* child, int* parent_int,
                            int* parent_leaf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int dsign = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(keys, n, i, i - dsign);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * dsign) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * dsign) > dmin) l += t;
  const int j = i + l * dsign;
  const int dnode = delta(keys, n, i, j);
  int s = 0;
  int t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, n, i, i + (s + t) * dsign) > dnode) s += t;
  } while (t > 1);
  const int gamma = i + s * dsign + (dsign < 0 ? -1 : 0);
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  const int left = (lo == gamma) ? ~gamma : gamma;
  const int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  child[i] = make_int2(left, right);
  if (left < 0) parent_leaf[~left] = i; else parent_int[left] = i;
  if (right < 0) parent_leaf[~right] = i; else parent_int[right] = i;
  if (i == 0) parent_int[0] = -1;
}

__device__ __forceinline__ void get_box(int c, const float4* __restrict__ leaf_box,
                                        const unsigned long long* __restrict__ keys, const float4* ibox,
                                        float4& lo, float4& hi) {
  if (c < 0) {
    const int prim = (int)(keys[~c] & 0xffffffffull);
    lo = leaf_box[2 * prim];
    hi = leaf_box[2 * prim + 1];
  } else {
    lo = __ldcg(ibox + 2 * c);  // L2-coherent: written by another thread of this kernel
    hi = __ldcg(ibox + 2 * c + 1);
  }
}

__global__ void k_refit(const float4* __restrict__ leaf_box, const unsigned long long* __restrict__ keys, int n,
                        const int2* __restrict__ child, const int* __restrict__ parent_int,
                        const int* __restrict__ parent_leaf, unsigned int* flags, float4* ibox, BvhNode* nodes) {
  const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
  if (leaf >= n) return;
  int node = parent_leaf[leaf];
  // a tree over unique 62-bit keys is at most 63 levels deep; the bound keeps
  // a malformed hierarchy from looping
  for (int guard = 0; node >= 0 && guard < 128; ++guard) {
    __threadfence();
    if (atomicAdd(&flags[node], 1u) == 0) return;  // the sibling's thread finishes this node
    __threadfence();
    const int2 ch = child[node];
    float4 llo, lhi, rlo, rhi;
    get_box(ch.x, leaf_box, keys, ibox, llo, lhi);
    get_box(ch.y, leaf_box, keys, ibox, rlo, rhi);
    const int lc = ch.x < 0 ? ~(int)(keys[~ch.x] & 0xffffffffull) : ch.x;
    const int rc = ch.y < 0 ? ~(int)(keys[~ch.y] & 0xffffffffull) : ch.y;
    BvhNode nd;
    nd.a = make_float4(llo.x, llo.y, llo.z, __int_as_float(lc));
    nd.b = make_float4(lhi.x, lhi.y, lhi.z, __int_as_float(rc));
    nd.c = make_float4(rlo.x, rlo.y, rlo.z, 0.0f);
    nd.d = make_float4(rhi.x, rhi.y, rhi.z, 0.0f);
    nodes[node] = nd;
    __stcg(ibox + 2 * node, make_float4(fminf(llo.x, rlo.x), fminf(llo.y, rlo.y), fminf(llo.z, rlo.z), 0.0f));
    __stcg(ibox + 2 * node + 1, make_float4(fmaxf(lhi.x, rhi.x), fmaxf(lhi.y, rhi.y), fmaxf(lhi.z, rhi.z), 0.0f));
    node = parent_int[node];
  }
}

}  // namespace

// d_box: [n][2] float4 (lo, hi) per primitive, already padded.
cudaError_t build_bvh(const float4* d_box, int n, const float lo[3], const float ext[3], BvhNode* d_nodes,
                      cudaStream_t st, std::string* err) {
  if (n < 2) return cudaSuccess;
  int npow = 1;
  while (npow < n) npow <<= 1;
  unsigned long long* keys = nullptr;
  int2* child = nullptr;
  int *pint = nullptr, *pleaf = nullptr;
  unsigned int* flags = nullptr;
  float4* ibox = nullptr;
  cudaError_t e = cudaSuccess;
  auto fail = [&](const char* what) {
    if (err) *err = std::string("BVH build: ") + what + ": " + cudaGetErrorString(e);
  };
  do {
    if ((e = cudaMallocAsync(&keys, sizeof(unsigned long long) * npow, st)) != cudaSuccess) { fail("alloc"); break; }
    if ((e = cudaMallocAsync(&child, sizeof(int2) * (n - 1), st)) != cudaSuccess) { fail("alloc"); break; }
    if ((e = cudaMallocAsync(&pint, sizeof(int) * (n - 1), st)) != cudaSuccess) { fail("alloc"); break; }
    if ((e = cudaMallocAsync(&pleaf, sizeof(int) * n, st)) != cudaSuccess) { fail("alloc"); break; }
    if ((e = cudaMallocAsync(&flags, sizeof(unsigned int) * (n - 1), st)) != cudaSuccess) { fail("alloc"); break; }
    if ((e = cudaMallocAsync(&ibox, sizeof(float4) * 2 * (n - 1), st)) != cudaSuccess) { fail("alloc"); break; }
    cudaMemsetAsync(flags, 0, sizeof(unsigned int) * (n - 1), st);
    const int TB = 256;
    const float ie[3] = {1.0f / ext[0], 1.0f / ext[1], 1.0f / ext[2]};
    const float emax = fmaxf(fmaxf(ext[0], ext[1]), ext[2]);
    k_morton<<<(npow + TB - 1) / TB, TB, 0, st>>>(d_box, n, npow, lo[0], lo[1], lo[2], ie[0], ie[1], ie[2],
                                                  0.5f * emax, keys);
    for (int k = 2; k <= npow; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) k_bitonic<<<(npow + TB - 1) / TB, TB, 0, st>>>(keys, npow, j, k);
    k_hierarchy<<<(n - 1 + TB - 1) / TB, TB, 0, st>>>(keys, n, child, pint, pleaf);
    k_refit<<<(n + TB - 1) / TB, TB, 0, st>>>(d_box, keys, n, child, pint, pleaf, flags, ibox, d_nodes);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail("launch"); break; }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { fail("run"); break; }
  } while (false);
  if (keys) cudaFreeAsync(keys, st);
  if (child) cudaFreeAsync(child, st);
  if (pint) cudaFreeAsync(pint, st);
  if (pleaf) cudaFreeAsync(pleaf, st);
  if (flags) cudaFreeAsync(flags, st);
  if (ibox) cudaFreeAsync(ibox, st);
  cudaStreamSynchronize(st);
  return e;
}

// ------------------------------------------------------------ SAH build
// Top-down surface-area-heuristic build on the host (MacDonald and Booth's cost
// model: a split of a node's primitives into L and R costs A(L) |L| + A(R) |R|,
// A the surface area of the side's bounding box).  Ranges of at most 64
// primitives try every split position in the centroid order along each axis;
// larger ones 32 equal-width centroid bins per axis (Wald, "On fast
// construction of SAH-based bounding volume hierarchies", 2007).  One
// primitive per leaf, so the tree has n - 1 internal nodes, like the LBVH, in
// the same node format; siblings get adjacent node numbers.  A range that
// could otherwise end deeper than kMaxDepth levels is split at its centroid
// median along the widest axis from there on, so no leaf lies deeper than
// kMaxDepth and the traversal stacks (48 entries) never overflow.
namespace {
struct HBox {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const HBox& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  double area() const {
    if (!(hi[0] >= lo[0])) return 0.0;
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return dx * dy + dy * dz + dz * dx;
  }
};
}  // namespace

bool build_bvh_sah(const std::vector<float4>& boxes, int n, std::vector<BvhNode>& nodes) {
  if (n < 2) return false;
  std::vector<HBox> pb(n);
  std::vector<float> cen(3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const float4 l = boxes[2 * i], h = boxes[2 * i + 1];
    pb[i].lo[0] = l.x; pb[i].lo[1] = l.y; pb[i].lo[2] = l.z;
    pb[i].hi[0] = h.x; pb[i].hi[1] = h.y; pb[i].hi[2] = h.z;
    for (int a = 0; a < 3; ++a) cen[3 * (size_t)i + a] = 0.5f * (pb[i].lo[a] + pb[i].hi[a]);
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  nodes.assign(n - 1, BvhNode{});
  struct Task {
    int begin, end, node, depth;
  };
  std::vector<Task> todo{{0, n, 0, 1}};
  int next = 1;
  constexpr int BINS = 32, EXACT = 64, kMaxDepth = 44;
  auto ceil_log2 = [](int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
  };
  std::vector<double> left_area(std::max(EXACT, BINS));
  while (!todo.empty()) {
    const Task t = todo.back();
    todo.pop_back();
    const int cnt = t.end - t.begin;
    int* r = idx.data() + t.begin;
    int mid = -1;
    if (t.depth + ceil_log2(cnt) >= kMaxDepth) {
      float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int k = 0; k < cnt; ++k)
        for (int a = 0; a < 3; ++a) {
          clo[a] = std::min(clo[a], cen[3 * (size_t)r[k] + a]);
          chi[a] = std::max(chi[a], cen[3 * (size_t)r[k] + a]);
        }
      int a = 0;
      for (int b = 1; b < 3; ++b)
        if (chi[b] - clo[b] > chi[a] - clo[a]) a = b;
      mid = cnt / 2;
      std::nth_element(r, r + mid, r + cnt, [&](int x, int y) {
        const float cx = cen[3 * (size_t)x + a], cy = cen[3 * (size_t)y + a];
        return cx < cy || (cx == cy && x < y);
      });
    } else if (cnt <= EXACT) {
      // every split position of the centroid order along each axis
      double best = INFINITY;
      int best_axis = -1, best_k = 0;
      for (int a = 0; a < 3; ++a) {
        std::sort(r, r + cnt, [&](int x, int y) {
          const float cx = cen[3 * (size_t)x + a], cy = cen[3 * (size_t)y + a];
          return cx < cy || (cx == cy && x < y);
        });
        HBox acc;
        for (int k = 0; k < cnt - 1; ++k) {
          acc.grow(pb[r[k]]);
          left_area[k] = acc.area() * (k + 1);
        }
        HBox racc;
        for (int k = cnt - 1; k >= 1; --k) {
          racc.grow(pb[r[k]]);
          const double c = left_area[k - 1] + racc.area() * (cnt - k);
          if (c < best) { best = c; best_axis = a; best_k = k; }
        }
      }
      const int a = best_axis;
      std::sort(r, r + cnt, [&](int x, int y) {
        const float cx = cen[3 * (size_t)x + a], cy = cen[3 * (size_t)y + a];
        return cx < cy || (cx == cy && x < y);
      });
      mid = best_k;
    } else {
      float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int k = 0; k < cnt; ++k)
        for (int a = 0; a < 3; ++a) {
          clo[a] = std::min(clo[a], cen[3 * (size_t)r[k] + a]);
          chi[a] = std::max(chi[a], cen[3 * (size_t)r[k] + a]);
        }
      double best = INFINITY;
      int best_axis = -1, best_bin = 0;
      for (int a = 0; a < 3; ++a) {
        const float ext = chi[a] - clo[a];
        if (!(ext > 0.0f)) continue;
        const float sc = (float)BINS / ext;
        HBox bb[BINS];
        int bc[BINS] = {};
        for (int k = 0; k < cnt; ++k) {
          const int b = std::min(BINS - 1, (int)((cen[3 * (size_t)r[k] + a] - clo[a]) * sc));
          bb[b].grow(pb[r[k]]);
          bc[b] += 1;
        }
        HBox acc;
        int nl = 0;
        for (int b = 0; b < BINS - 1; ++b) {
          acc.grow(bb[b]);
          nl += bc[b];
          left_area[b] = acc.area() * nl;
        }
        HBox racc;
        int nr = 0;
        for (int b = BINS - 1; b >= 1; --b) {
          racc.grow(bb[b]);
          nr += bc[b];
          if (nr == 0 || nr == cnt) continue;
          const double c = left_area[b - 1] + racc.area() * nr;
          if (c < best) { best = c; best_axis = a; best_bin = b; }
        }
      }
      if (best_axis >= 0) {
        const int a = best_axis;
        const float sc = (float)BINS / (chi[a] - clo[a]);
        int* m = std::partition(r, r + cnt, [&](int x) {
          return std::min(BINS - 1, (int)((cen[3 * (size_t)x + a] - clo[a]) * sc)) < best_bin;
        });
        mid = (int)(m - r);
      }
      if (mid <= 0 || mid >= cnt) {
        // all centroids in one bin: the median of the index order
        std::sort(r, r + cnt);
        mid = cnt / 2;
      }
    }
    HBox side[2];
    int child[2];
    const int rng[2][2] = {{0, mid}, {mid, cnt}};
    for (int sdx = 0; sdx < 2; ++sdx) {
      for (int k = rng[sdx][0]; k < rng[sdx][1]; ++k) side[sdx].grow(pb[r[k]]);
      if (rng[sdx][1] - rng[sdx][0] == 1) {
        child[sdx] = ~r[rng[sdx][0]];
      } else {
        child[sdx] = next++;
      }
    }
    for (int sdx = 1; sdx >= 0; --sdx)
      if (child[sdx] >= 0) todo.push_back({t.begin + rng[sdx][0], t.begin + rng[sdx][1], child[sdx], t.depth + 1});
    BvhNode& nd = nodes[t.node];
    float cw[2];
    std::memcpy(cw, child, sizeof(cw));
    nd.a = make_float4(side[0].lo[0], side[0].lo[1], side[0].lo[2], cw[0]);
    nd.b = make_float4(side[0].hi[0], side[0].hi[1], side[0].hi[2], cw[1]);
    nd.c = make_float4(side[1].lo[0], side[1].lo[1], side[1].lo[2], 0.0f);
    nd.d = make_float4(side[1].hi[0], side[1].hi[1], side[1].hi[2], 0.0f);
  }
  return next == n - 1;
}

}  // namespace mars
