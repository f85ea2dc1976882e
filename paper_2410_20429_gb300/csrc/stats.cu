// stats.cu -- image statistics and the fixed-point count update.
//
// Image statistics (Sec. 4.1, "Image estimates"): the iteration's one-sample
// image is added to the running sum; the pixel estimate is a 3x3 box filter of
// the running mean over in-image neighbours, floored at 1e-3 x the channel mean
// (the paper denoises with OIDN instead); V_I is the mean over pixels and
// channels of ((min(I, outlier x est) - est) / est)^2 ("Outlier clamping");
// C_I is rays per pixel.
//
// Update (Eq. "optimalBeta", spatial form of Sec. 3.1 "Optimization"): per
// cell, technique and channel, the moments and the ratio in float64 (the square
// roots in float32),
//   q^RR = sqrt(C_I / C_t * m2 / V_I),   q^S = sqrt(C_I / C_t * var / V_I),
// with m2, var the per-sample moments of Sec. 4.1 "Local estimates" and C_t the
// mean cost; cells with n < 2 or no cost keep their factors; statistics reset.
// The guided technique's per-cell CDF is rebuilt from the accumulated deposits.
#include <algorithm>

#include "device.cuh"

namespace mars {

namespace {

constexpr int IMG_THREADS = 256;

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;  // valid in thread 0
}

// The RGB of a warp's 32 consecutive pixels [b, b + 32) -- lane l holds pixel
// b + l -- written to a packed float RGB image as 24 aligned 16-byte stores of
// the 384 bytes instead of 96 scattered 4-byte stores.  A page-locked host
// image is written by this pass across the chip-to-chip link, where partial
// writes cost far more than whole ones.  A partial warp, or an output that is
// not 16-byte aligned, stores per channel.  `stage`: this warp's 96 floats of
// shared memory.  b, npix and out are uniform over the warp.
__device__ __forceinline__ void store_rgb_warp(float* __restrict__ out, int b, int npix, float x, float y, float z,
                                               float* stage) {
  const int lane = threadIdx.x & 31;
  if (b + 32 <= npix && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    stage[3 * lane] = x;
    stage[3 * lane + 1] = y;
    stage[3 * lane + 2] = z;
    __syncwarp();
    if (lane < 24)
      reinterpret_cast<float4*>(out + 3 * (size_t)b)[lane] = reinterpret_cast<const float4*>(stage)[lane];
    __syncwarp();
  } else if (b + lane < npix) {
    const size_t q = 3 * (size_t)(b + lane);
    out[q] = x;
    out[q + 1] = y;
    out[q + 2] = z;
  }
}

// sum of a float over the warp (every lane receives it)
__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// image sums in the statistics' precision: float64, or float32 for the
// float32-statistics variant
template <typename T>
__device__ __forceinline__ void add_sum(double* d64, float* d32, T v);
template <>
__device__ __forceinline__ void add_sum<double>(double* d64, float*, double v) { atomicAdd(d64, v); }
template <>
__device__ __forceinline__ void add_sum<float>(double*, float* d32, float v) { atomicAdd(d32, v); }

// The channel sums only set the estimate's floor: each warp sums its pixels in
// float32, the block adds its warps' sums in T (a float64 operation per warp
// instead of per pixel: float64 runs at 1/64 of the float32 rate here).
template <typename T>
__global__ void __launch_bounds__(IMG_THREADS) k_img_accum(DevCache c, int npix, const IterArgs* __restrict__ itp,
                                                            float* out) {
  __shared__ T sh[3][IMG_THREADS / 32];
  __shared__ __align__(16) float stage[IMG_THREADS * 3];
  if (c.ctr->any_overflow) return;
  const int n_prev = itp->n_prev;
  const float inv = 1.0f / (float)(n_prev + 1);
  float m0 = 0.f, m1 = 0.f, m2 = 0.f;
  // warp-uniform trip count: the warp stores its pixels together
  for (int b = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < npix; b += gridDim.x * blockDim.x) {
    const int p = b + (threadIdx.x & 31);
    float4 I = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p < npix) {
      I = c.img[p];
      float4 rs = c.run_sum[p];
      rs.x += I.x; rs.y += I.y; rs.z += I.z;
      c.run_sum[p] = rs;
      m0 += rs.x * inv;
      m1 += rs.y * inv;
      m2 += rs.z * inv;
    }
    if (out) store_rgb_warp(out, b, npix, I.x, I.y, I.z, stage + 96 * (threadIdx.x >> 5));
  }
  m0 = warp_sum(m0);
  m1 = warp_sum(m1);
  m2 = warp_sum(m2);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = (T)m0;
    sh[1][w] = (T)m1;
    sh[2][w] = (T)m2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T s0 = 0, s1 = 0, s2 = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s0 += sh[0][k];
      s1 += sh[1][k];
      s2 += sh[2][k];
    }
    const int slot = blockIdx.x % IMG_SLOTS;
    add_sum<T>(&c.ctr->img_part[slot][0], &c.ctr->img_part32[slot][0], s0);
    add_sum<T>(&c.ctr->img_part[slot][1], &c.ctr->img_part32[slot][1], s1);
    add_sum<T>(&c.ctr->img_part[slot][2], &c.ctr->img_part32[slot][2], s2);
  }
}

// Sum of the squared relative errors of one pixel's three channels, in
// float32 with every operation rounded on its own (no contraction), so that the
// brightest-pixel rejection subtracts exactly the term that was added; with
// `clamp` the sample is first bounded at outlier x estimate.
__device__ __forceinline__ float pixel_err(float4 I, float e0, float e1, float e2, float outlier, bool clamp) {
  const float i0 = clamp ? fminf(I.x, outlier * e0) : I.x;
  const float i1 = clamp ? fminf(I.y, outlier * e1) : I.y;
  const float i2 = clamp ? fminf(I.z, outlier * e2) : I.z;
  const float r0 = __fdiv_rn(__fsub_rn(i0, e0), e0);
  const float r1 = __fdiv_rn(__fsub_rn(i1, e1), e1);
  const float r2 = __fdiv_rn(__fsub_rn(i2, e2), e2);
  return __fadd_rn(__fadd_rn(__fmul_rn(r0, r0), __fmul_rn(r1, r1)), __fmul_rn(r2, r2));
}

template <typename T>
__global__ void __launch_bounds__(IMG_THREADS) k_img_est(DevCache c, int W, int H, const IterArgs* __restrict__ itp) {
  __shared__ T sh[IMG_THREADS / 32];
  if (c.ctr->any_overflow) return;
  const int n_prev = itp->n_prev;
  const float outlier = itp->outlier;
  const bool clamp = itp->drop_k <= 0;  // the brightest-pixel rejection replaces the clamp
  const int npix = W * H;
  const float inv = 1.0f / (float)(n_prev + 1);
  const bool f32 = c.stats32 != nullptr;
  // the floor: 1e-3 x each channel's mean, its sum added over the slots in the
  // statistics' precision by the first warp
  __shared__ float fl_sh[3];
  if (threadIdx.x < 32) {
    static_assert(IMG_SLOTS == 32, "one slot per lane");
    T ch[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T v = f32 ? (T)c.ctr->img_part32[threadIdx.x][q] : (T)c.ctr->img_part[threadIdx.x][q];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      ch[q] = v;
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < 3; ++q) fl_sh[q] = 1e-3f * (float)(ch[q] / (T)npix);
  }
  __syncthreads();
  const float fl0 = fl_sh[0], fl1 = fl_sh[1], fl2 = fl_sh[2];
  T vi = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const int x = p % W, y = p / W;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    int k = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx, yy = y + dy;
        if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
        const float4 r = c.run_sum[yy * W + xx];
        s0 += r.x * inv;
        s1 += r.y * inv;
        s2 += r.z * inv;
        ++k;
      }
    float e0 = fmaxf(fmaxf(s0 / (float)k, fl0), 1e-8f);
    float e1 = fmaxf(fmaxf(s1 / (float)k, fl1), 1e-8f);
    float e2 = fmaxf(fmaxf(s2 / (float)k, fl2), 1e-8f);
    c.est[p] = make_float4(e0, e1, e2, 0.0f);
    vi += (T)pixel_err(c.img[p], e0, e1, e2, outlier, clamp);
  }
  vi = block_sum<T>(vi, sh);
  const int slot = blockIdx.x % IMG_SLOTS;
  if (threadIdx.x == 0) add_sum<T>(&c.ctr->img_part[slot][3], &c.ctr->img_part32[slot][3], vi);
}

__global__ void __launch_bounds__(IMG_THREADS) k_img_copy(DevCache c, int npix, float* out) {
  __shared__ __align__(16) float stage[IMG_THREADS * 3];
  if (c.ctr->any_overflow) return;
  for (int b = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < npix; b += gridDim.x * blockDim.x) {
    const int p = b + (threadIdx.x & 31);
    const float4 I = p < npix ? c.img[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    store_rgb_warp(out, b, npix, I.x, I.y, I.z, stage + 96 * (threadIdx.x >> 5));
  }
}

// the pixels of one range of the frame (a shard of a multi-GPU job), one
// thread per pixel: three scalar stores, since a range need not start on a
// warp-aligned pixel
__global__ void __launch_bounds__(IMG_THREADS) k_img_copy_range(DevCache c, int p0, int p1, float* out) {
  if (c.ctr->any_overflow) return;
  for (int p = p0 + blockIdx.x * blockDim.x + threadIdx.x; p < p1; p += gridDim.x * blockDim.x) {
    const float4 I = c.img[p];
    out[3 * (size_t)p] = I.x;
    out[3 * (size_t)p + 1] = I.y;
    out[3 * (size_t)p + 2] = I.z;
  }
}

// ---- brightest-pixel rejection of V_I (Sec. 5.1 "Implementation")
// Brightness order: float32 luminance (products and sums rounded one by one,
// as the oracle does), descending, then pixel index ascending; the key is
// unique per pixel and 0 never names one.
__device__ __forceinline__ unsigned long long bright_key(float4 I, int p) {
  float l = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, I.x), __fmul_rn(0.7152f, I.y)), __fmul_rn(0.0722f, I.z));
  if (!(l > 0.0f)) l = 0.0f;
  return ((unsigned long long)__float_as_uint(l) << 32) | (unsigned long long)(0xffffffffu - (unsigned)p);
}

// The K largest keys seen: L descending and zero-filled (entries from K on stay
// 0), kth = L[K - 1], so that a key that cannot enter is rejected by one
// comparison.
struct TopK {
  unsigned long long L[MAX_DROP];
  unsigned long long kth;
};

__device__ __forceinline__ void topk_clear(TopK& t) {
#pragma unroll
  for (int q = 0; q < MAX_DROP; ++q) t.L[q] = 0;
  t.kth = 0;
}

__device__ __forceinline__ void topk_insert(TopK& t, int K, unsigned long long x) {
  if (x <= t.kth) return;
  unsigned long long kth = 0;
#pragma unroll
  for (int q = 0; q < MAX_DROP; ++q) {
    if (q < K && x > t.L[q]) {
      const unsigned long long v = t.L[q];
      t.L[q] = x;
      x = v;
    }
    if (q == K - 1) kth = t.L[q];
  }
  t.kth = kth;
}

// largest of a key over the warp (every lane receives it)
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}

// K rounds of "largest head of all threads' lists": the owner pops it; out[r]
// (thread 0) receives the r-th largest key of the block (0 if none).  sh holds
// one key per warp (at most 32 warps).
__device__ __forceinline__ void topk_block(TopK& t, int K, unsigned long long* out, unsigned long long* sh,
                                           unsigned long long* best) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int r = 0; r < K; ++r) {
    const unsigned long long v = warp_max_key(t.L[0]);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
      const unsigned long long m = warp_max_key(lane < nw ? sh[lane] : 0ull);
      if (lane == 0) {
        *best = m;
        out[r] = m;
      }
    }
    // sh is rewritten, and *best written, only after the next round's first
    // barrier, which every thread reaches after reading *best here
    __syncthreads();
    const unsigned long long m = *best;
    if (m != 0 && t.L[0] == m) {
#pragma unroll
      for (int q = 0; q < MAX_DROP - 1; ++q) t.L[q] = t.L[q + 1];
      t.L[MAX_DROP - 1] = 0;
    }
  }
}

// block b: the K brightest pixels of its contiguous pixel range
__global__ void __launch_bounds__(IMG_THREADS) k_img_topk(DevCache c, int npix, const IterArgs* __restrict__ itp) {
  __shared__ unsigned long long sh[IMG_THREADS / 32], best;
  if (c.ctr->any_overflow) return;
  const int K = itp->drop_k;
  if (K <= 0) return;
  const int per = (npix + (int)gridDim.x - 1) / (int)gridDim.x;
  const int lo = (int)blockIdx.x * per, hi = min(npix, lo + per);
  TopK t;
  topk_clear(t);
  for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) topk_insert(t, K, bright_key(c.img[p], p));
  topk_block(t, K, c.topk + (size_t)blockIdx.x * K, sh, &best);
}

// one block: the K brightest of all candidates leave the V_I sum (their terms,
// recomputed from the same image and estimate, are subtracted)
template <typename T>
__global__ void __launch_bounds__(1024) k_img_drop(DevCache c, int nblocks, const IterArgs* __restrict__ itp) {
  __shared__ unsigned long long sh[32], best, sel[MAX_DROP];
  if (c.ctr->any_overflow) return;
  const int K = itp->drop_k;
  if (K <= 0) return;
  TopK t;
  topk_clear(t);
  const int ncand = nblocks * K;  // k_img_topk wrote K keys per block
  for (int i = threadIdx.x; i < ncand; i += blockDim.x) topk_insert(t, K, c.topk[i]);
  topk_block(t, K, sel, sh, &best);
  if (threadIdx.x == 0) {
    T sum = 0;
    int n = 0;
    for (int r = 0; r < K; ++r) {
      if (sel[r] == 0) continue;
      const int p = (int)(0xffffffffu - (unsigned)(sel[r] & 0xffffffffull));
      const float4 e = c.est[p];
      sum += (T)pixel_err(c.img[p], e.x, e.y, e.z, 0.0f, false);
      ++n;
    }
    if (c.stats32) c.ctr->vi_sum32 -= (float)sum; else c.ctr->vi_sum -= (double)sum;
    c.ctr->vi_dropped = n;
  }
}

// ---- progressive combination (Sec. 5.1): weight 1 / V_I of this iteration
__global__ void __launch_bounds__(IMG_THREADS) k_img_combine(DevCache c, int npix, const IterArgs* __restrict__ itp) {
  if (c.ctr->any_overflow) return;
  const int mode = itp->combine;
  if (mode == 0) return;
  const float w = (float)(1.0 / fmax(c.ctr->VI, 1e-12));
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const float4 I = c.img[p];
    float4 a = mode == 2 ? make_float4(0.f, 0.f, 0.f, 0.f) : c.comb[p];
    a.x += w * I.x;
    a.y += w * I.y;
    a.z += w * I.z;
    c.comb[p] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *c.comb_w = (mode == 2 ? 0.0 : *c.comb_w) + (double)w;
}

__global__ void __launch_bounds__(IMG_THREADS) k_img_comb_out(DevCache c, int npix, float* out) {
  __shared__ __align__(16) float stage[IMG_THREADS * 3];
  const double w = *c.comb_w;
  const float inv = w > 0.0 ? (float)(1.0 / w) : 0.0f;
  for (int b = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < npix; b += gridDim.x * blockDim.x) {
    const int p = b + (threadIdx.x & 31);
    const float4 a = p < npix ? c.comb[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    store_rgb_warp(out, b, npix, a.x * inv, a.y * inv, a.z * inv, stage + 96 * (threadIdx.x >> 5));
  }
}

// V_I and C_I of the training iteration the update closes: the means over its
// iterations (Sec. 4.1 "Image estimates" averages the squared relative errors
// over every sample of the iteration); 0 when no image statistics ran, which
// keeps every factor
__device__ __forceinline__ void image_means(const DevCache& c, double& VI, double& CI) {
  const double n = c.img_acc[2];
  VI = n > 0.0 ? c.img_acc[0] / n : 0.0;
  CI = n > 0.0 ? c.img_acc[1] / n : 0.0;
}

// one warp: V_I and C_I from the slots' sums (and the rejection's subtraction)
__global__ void k_img_final(DevCache c, int npix) {
  if (c.ctr->any_overflow) return;
  double v64 = c.ctr->img_part[threadIdx.x][3];
  float v32 = c.ctr->img_part32[threadIdx.x][3];
  for (int off = 16; off > 0; off >>= 1) {
    v64 += __shfl_xor_sync(0xffffffffu, v64, off);
    v32 += __shfl_xor_sync(0xffffffffu, v32, off);
  }
  if (threadIdx.x != 0) return;
  c.ctr->vi_sum += v64;
  c.ctr->vi_sum32 += v32;
  const int kept = npix - c.ctr->vi_dropped;  // V_I: the mean over the pixels that were kept
  if (c.stats32) {
    c.ctr->VI = (double)(c.ctr->vi_sum32 / (3.0f * (float)kept));
    c.ctr->CI = (double)((float)c.ctr->rays / (float)npix);
  } else {
    c.ctr->VI = c.ctr->vi_sum / (3.0 * (double)kept);
    c.ctr->CI = (double)c.ctr->rays / (double)npix;
  }
  // a training iteration of several such iterations: the update averages them
  c.img_acc[0] += c.ctr->VI;
  c.img_acc[1] += c.ctr->CI;
  c.img_acc[2] += 1.0;
}

__global__ void k_update_counts(DevCache c) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c.n_cells * NT) return;
  const int t = idx % NT;
  // structure of arrays: statistic k of entry idx at stats[k * plane + idx]
  const size_t plane = (size_t)c.n_cells * NT;
  double* sp = c.stats + idx;
  const double n = sp[0];
  // no sample landed in this (cell, technique): every sum is already zero
  if (n == 0.0) return;
  double v[NSTAT];
#pragma unroll
  for (int k = 1; k < NSTAT; ++k) v[k] = sp[k * plane];
  double VI, CI;
  image_means(c, VI, CI);
  const double cost = v[7];
  if (slot_on(c.techniques, t) && VI > 1e-12 && n >= 2.0 && cost > 0.0) {
    // C_I / C_t / V_I with C_t = cost / n, and 1 / n, formed once in float64
    const double inv_n = 1.0 / n;
    const double r = CI * n / (cost * VI);
    const double s1[3] = {v[1], v[2], v[3]}, s2v[3] = {v[4], v[5], v[6]};
    float qr[3], qs[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const double m1 = s1[ch] * inv_n, m2 = s2v[ch] * inv_n;
      double var = m2 - m1 * m1;
      if (var < 0.0) var = 0.0;
      // square roots in float32 of the float64 products (the factors are stored
      // in float32; a float64 square root costs tens of operations at 1/64 of
      // the float32 rate on this part): within 1e-7 of the float64 root
      qr[ch] = sqrtf((float)(r * m2));
      qs[ch] = sqrtf((float)(r * var));
    }
    c.cnt[2 * idx] = make_float4(qr[0], qr[1], qr[2], 1.0f);
    c.cnt[2 * idx + 1] = make_float4(qs[0], qs[1], qs[2], 0.0f);
  }
#pragma unroll
  for (int k = 0; k < NSTAT; ++k) sp[k * plane] = 0.0;
}

// the same update with float32 statistics and arithmetic (precision study)
__global__ void k_update_counts32(DevCache c) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c.n_cells * NT) return;
  const int t = idx % NT;
  float4* s4 = reinterpret_cast<float4*>(c.stats32 + (size_t)idx * NSTAT);
  const float4 a = s4[0];
  if (a.x == 0.0f) return;
  const float4 b = s4[1];
  double VI64, CI64;
  image_means(c, VI64, CI64);
  const float VI = (float)VI64, CI = (float)CI64;
  const float n = a.x, cost = b.w;
  if (slot_on(c.techniques, t) && VI > 1e-12f && n >= 2.0f && cost > 0.0f) {
    const float inv_n = 1.0f / n;
    const float r = CI * n / (cost * VI);
    const float s1[3] = {a.y, a.z, a.w}, s2v[3] = {b.x, b.y, b.z};
    float qr[3], qs[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float m1 = s1[ch] * inv_n, m2 = s2v[ch] * inv_n;
      float var = m2 - m1 * m1;
      if (var < 0.0f) var = 0.0f;
      qr[ch] = sqrtf(r * m2);
      qs[ch] = sqrtf(r * var);
    }
    c.cnt[2 * idx] = make_float4(qr[0], qr[1], qr[2], 1.0f);
    c.cnt[2 * idx + 1] = make_float4(qs[0], qs[1], qs[2], 0.0f);
  }
  s4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  s4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---- float-float arithmetic: a value held as an unevaluated sum hi + lo of two
// floats, about 48 significant bits, from float32 operations only (float64 runs
// at 1/64 of the float32 rate on this part).  TwoSum (Knuth), FastTwoSum
// (Dekker, |a| >= |b|) and TwoProduct through a fused multiply-add (Ogita, Rump
// and Oishi 2005); addition, product and quotient as in the double-double
// arithmetic of Hida, Li and Bailey (2001).
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.hi, b.hi);
  const FF t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }
// a x b for a float b
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, e));
}
// a / b, b > 0: the float quotient of the leading parts, corrected twice by the
// remainder
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  FF r = ff_add(a, ff_neg(ff_mul_f(b, q1)));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  r = ff_add(r, ff_neg(ff_mul_f(b, q2)));
  const float q3 = __fdiv_rn(r.hi, b.hi);
  const FF q = fast_two_sum(q1, q2);
  return ff_add(q, FF{q3, 0.0f});
}
__device__ __forceinline__ FF ff_shfl_xor(FF a, int off) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}
__device__ __forceinline__ FF ff_shfl_up(FF a, int off) {
  return {__shfl_up_sync(0xffffffffu, a.hi, off), __shfl_up_sync(0xffffffffu, a.lo, off)};
}
// a float-float constant from a double one (folded at compile time)
#define FF_CONST(x) FF{(float)(x), (float)((x) - (double)(float)(x))}

// one warp per cell: P_b = 0.9 h_b / H + 0.1 / 256 (uniform when H = 0), then an
// inclusive prefix sum, in float-float arithmetic (every step of the float64
// formulation, at about 48 bits; each CDF value is rounded once to float32).
// Lane l holds bins 8 l .. 8 l + 7 (two float4 loads and stores).  Only cells
// that received deposits since their last rebuild are rebuilt: the others' CDF
// already is the one their histogram gives.
__global__ void k_guide_update(DevCache c) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= c.n_cells || !c.guide_dirty[warp]) return;
  __syncwarp();
  if (lane == 0) c.guide_dirty[warp] = 0;
  const float4* h = reinterpret_cast<const float4*>(c.guide_hist + (size_t)warp * GUIDE_BINS) + 2 * lane;
  float4* cdf = reinterpret_cast<float4*>(c.guide_cdf + (size_t)warp * GUIDE_BINS) + 2 * lane;
  const float4 h0 = h[0], h1 = h[1];
  const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
  FF H{hv[0], 0.0f};
#pragma unroll
  for (int k = 1; k < 8; ++k) H = ff_add(H, FF{hv[k], 0.0f});
  for (int off = 16; off > 0; off >>= 1) H = ff_add(H, ff_shfl_xor(H, off));
  // every lane takes lane 0's total (the butterfly's lanes add in other orders)
  H = FF{__shfl_sync(0xffffffffu, H.hi, 0), __shfl_sync(0xffffffffu, H.lo, 0)};
  const bool pos = H.hi > 0.0f;
  const FF sc = pos ? ff_div(FF_CONST(0.9), H) : FF{0.0f, 0.0f};
  const FF base = pos ? FF_CONST(0.1 / GUIDE_BINS) : FF_CONST(1.0 / GUIDE_BINS);
  FF v[8];
  FF run{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = ff_add(ff_mul_f(sc, hv[k]), base);
    run = ff_add(run, v[k]);
  }
  FF incl = run;
  for (int off = 1; off < 32; off <<= 1) {
    const FF y = ff_shfl_up(incl, off);
    if (lane >= off) incl = ff_add(incl, y);
  }
  FF acc = ff_add(incl, ff_neg(run));
  float o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    acc = ff_add(acc, v[k]);
    o[k] = __fadd_rn(acc.hi, acc.lo);
  }
  if (lane == 31) o[7] = 1.0f;
  cdf[0] = make_float4(o[0], o[1], o[2], o[3]);
  cdf[1] = make_float4(o[4], o[5], o[6], o[7]);
}
#undef FF_CONST

// samples of the iteration per octree leaf, all techniques (exact in float32
// below 2^24), read before the update zeroes the statistics
__global__ void k_leaf_samples(DevCache c) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= c.oct_meta[1]) return;
  float n = 0.0f;
  const size_t plane = (size_t)c.n_cells * NT;
#pragma unroll
  for (int t = 0; t < NT; ++t)
    n += c.stats32 ? c.stats32[((size_t)L * NT + t) * NSTAT] : (float)c.stats[(size_t)L * NT + t + 0 * plane];
  c.oct_leaf_n[L] = n;
}

// Octree refinement (one block): leaves in cell order whose samples reached
// split_samples and whose level is below OCT_LMAX split into 8 while the leaf
// count stays within n_cells.  Split s turns the leaf's node into an internal
// node with children at nodes + 8 s; octant 0 keeps the cell, octant o > 0
// gets the new cell leaves + 7 s + o - 1.  The order, and hence the numbering,
// comes from a block-wide exclusive scan: deterministic.
constexpr int REFINE_THREADS = 1024;
__global__ void __launch_bounds__(REFINE_THREADS) k_octree_refine(DevCache c) {
  __shared__ int wsum[REFINE_THREADS / 32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nn = c.oct_meta[0], nl = c.oct_meta[1];
  int budget = (c.n_cells - nl) / 7;
  const int bn = (c.oct_cap_nodes - nn) / 8;
  if (bn < budget) budget = bn;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int L0 = 0; L0 < nl; L0 += REFINE_THREADS) {
    const int L = L0 + tid;
    const int flag = (L < nl && c.oct_leaf_n[L] >= c.split_samples && c.oct_leaf_level[L] < OCT_LMAX) ? 1 : 0;
    int incl = flag;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int v = wsum[lane];
      int wi = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += y;
      }
      wsum[lane] = wi - v;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    const int s = s_base + wsum[warp] + incl - flag;
    if (flag && s < budget) {
      const int base = nn + 8 * s;
      c.oct_nodes[c.oct_leaf_node[L]] = base;
      c.oct_nodes[base] = ~L;
      c.oct_leaf_node[L] = base;
      const int lev = c.oct_leaf_level[L] + 1;
      c.oct_leaf_level[L] = lev;
      for (int o = 1; o < 8; ++o) {
        const int cn = nl + 7 * s + o - 1;
        c.oct_nodes[base + o] = ~cn;
        c.oct_leaf_node[cn] = base + o;
        c.oct_leaf_level[cn] = lev;
      }
      c.oct_split[s] = L;
    }
    __syncthreads();
    if (tid == REFINE_THREADS - 1) s_base += wsum[warp] + incl;  // the pass's total
    __syncthreads();
  }
  if (tid == 0) {
    const int splits = s_base < budget ? s_base : budget;
    c.oct_meta[0] = nn + 8 * splits;
    c.oct_meta[1] = nl + 7 * splits;
    c.oct_meta[2] = splits;
  }
}

// children of this refinement inherit their parent's counts and guide
// histogram and CDF (one thread per child)
__global__ void k_octree_inherit(DevCache c) {
  const int splits = c.oct_meta[2];
  const int nl0 = c.oct_meta[1] - 7 * splits;
  const bool guided = c.techniques & MARS_TECH_GUIDED;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 7 * splits; k += gridDim.x * blockDim.x) {
    const int s = k / 7, o = k % 7 + 1;
    const int L = c.oct_split[s], cn = nl0 + 7 * s + o - 1;
#pragma unroll
    for (int q = 0; q < 2 * NT; ++q) c.cnt[(size_t)cn * 2 * NT + q] = c.cnt[(size_t)L * 2 * NT + q];
    if (guided) {
      const float4* hs = reinterpret_cast<const float4*>(c.guide_hist + (size_t)L * GUIDE_BINS);
      const float4* cs = reinterpret_cast<const float4*>(c.guide_cdf + (size_t)L * GUIDE_BINS);
      float4* hd = reinterpret_cast<float4*>(c.guide_hist + (size_t)cn * GUIDE_BINS);
      float4* cd = reinterpret_cast<float4*>(c.guide_cdf + (size_t)cn * GUIDE_BINS);
      for (int q = 0; q < GUIDE_BINS / 4; ++q) {
        hd[q] = hs[q];
        cd[q] = cs[q];
      }
      c.guide_dirty[cn] = 0;
    }
  }
}

}  // namespace

cudaError_t launch_leaf_samples(const DevCache& c, cudaStream_t st) {
  k_leaf_samples<<<(c.n_cells + 255) / 256, 256, 0, st>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_octree_refine(const DevCache& c, int num_sms, cudaStream_t st) {
  k_octree_refine<<<1, REFINE_THREADS, 0, st>>>(c);
  k_octree_inherit<<<num_sms, 128, 0, st>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_image_stats(const DevCache& c, int width, int height, const IterArgs* it,
                               float* image_out_dev, bool drop, bool combine, int num_sms, cudaStream_t st) {
  const int npix = width * height;
  int blocks = (npix + IMG_THREADS - 1) / IMG_THREADS;
  // four blocks per SM, grid-stride beyond: fewer blocks, fewer float64 atomics
  // (measured: 1024^2 image pass 0.19 -> 0.10 ms against one block per 256 pixels)
  const int cap = 4 * std::max(num_sms, 1);
  if (blocks > cap) blocks = cap;
  const int tblocks = std::min(blocks, IMG_TOPK_BLOCKS);
  if (c.stats32) {
    k_img_accum<float><<<blocks, IMG_THREADS, 0, st>>>(c, npix, it, image_out_dev);
    k_img_est<float><<<blocks, IMG_THREADS, 0, st>>>(c, width, height, it);
  } else {
    k_img_accum<double><<<blocks, IMG_THREADS, 0, st>>>(c, npix, it, image_out_dev);
    k_img_est<double><<<blocks, IMG_THREADS, 0, st>>>(c, width, height, it);
  }
  if (drop) {
    // candidates: tblocks x drop_k keys (drop_k <= MAX_DROP; the buffer holds
    // IMG_TOPK_BLOCKS x MAX_DROP)
    k_img_topk<<<tblocks, IMG_THREADS, 0, st>>>(c, npix, it);
    if (c.stats32)
      k_img_drop<float><<<1, 1024, 0, st>>>(c, tblocks, it);
    else
      k_img_drop<double><<<1, 1024, 0, st>>>(c, tblocks, it);
  }
  k_img_final<<<1, IMG_SLOTS, 0, st>>>(c, npix);
  if (combine) k_img_combine<<<blocks, IMG_THREADS, 0, st>>>(c, npix, it);
  return cudaGetLastError();
}

cudaError_t launch_combined_out(const DevCache& c, int npix, float* out, cudaStream_t st) {
  int blocks = (npix + IMG_THREADS - 1) / IMG_THREADS;
  if (blocks > 4096) blocks = 4096;
  k_img_comb_out<<<blocks, IMG_THREADS, 0, st>>>(c, npix, out);
  return cudaGetLastError();
}

cudaError_t launch_image_copy(const DevCache& c, int npix, float* out, cudaStream_t st) {
  int blocks = (npix + IMG_THREADS - 1) / IMG_THREADS;
  if (blocks > 4096) blocks = 4096;
  k_img_copy<<<blocks, IMG_THREADS, 0, st>>>(c, npix, out);
  return cudaGetLastError();
}

cudaError_t launch_image_copy_range(const DevCache& c, int p0, int p1, float* out, cudaStream_t st) {
  int blocks = (p1 - p0 + IMG_THREADS - 1) / IMG_THREADS;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_img_copy_range<<<blocks, IMG_THREADS, 0, st>>>(c, p0, p1, out);
  return cudaGetLastError();
}

cudaError_t launch_update(const DevCache& c, int num_sms, cudaStream_t st) {
  (void)num_sms;
  const int n = c.n_cells * NT;
  if (c.stats32)
    k_update_counts32<<<(n + 255) / 256, 256, 0, st>>>(c);
  else
    k_update_counts<<<(n + 255) / 256, 256, 0, st>>>(c);
  if (c.techniques & MARS_TECH_GUIDED) k_guide_update<<<(c.n_cells * 32 + 255) / 256, 256, 0, st>>>(c);
  return cudaGetLastError();
}

}  // namespace mars
