// static_scratch.cu -- mars_image_stats_static: the image-statistics pass of
// one iteration for callers that cannot allocate device memory.
//
// Its only scratch (per-row partial sums of a deterministic two-level
// reduction) lives in the file-scope device array g_row_sums below; the caller
// passes every input and output.  The array holds kMaxRows rows, so images up
// to kMaxRows rows high are accepted and taller ones are rejected.  Every call
// on a device shares the array: each call rewrites every slot it reads before
// reading it, so nothing depends on what an earlier call left there, but calls
// whose work overlaps on the GPU (different streams, or a second call before
// the first finished on another stream) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "abi_internal.h"

namespace {

constexpr int kMaxRows = 8192;
constexpr int kSlotsPerRow = 4;  // running-mean sum per channel, V_I partial
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// rows x slots of float64 partial sums, then 4 slots of totals
static __device__ __align__(256) double g_row_sums[kMaxRows * kSlotsPerRow + 4];

std::mutex g_setup_mutex;
double* g_scratch_of_device[kMaxDevices] = {};

// Device address of g_row_sums on the current device.  Host code must not use
// the symbol itself (it names a host-side stand-in), so the address is looked
// up once per device with that device current and cached for the life of the
// process.  A cudaDeviceReset (or a host that tears down the device's primary
// context) invalidates the cached address; the entry point must not be used on
// that device afterwards.
mars_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return mars::set_error(MARS_ERR_CUDA, "no current CUDA device");
  if (dev < 0 || dev >= kMaxDevices)
    return mars::set_error(MARS_ERR_INVALID_ARG, "device %d beyond the %d supported", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  if (!g_scratch_of_device[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_row_sums);
    if (e != cudaSuccess || !p)
      return mars::set_error(MARS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                             cudaGetErrorString(e));
    g_scratch_of_device[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_of_device[dev];
  return MARS_OK;
}

// fixed-order tree reduction over a block (deterministic)
__device__ __forceinline__ double block_reduce(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// run_sum += image; per row, the sums of the running mean per channel
__global__ void __launch_bounds__(kThreads) k_rows_accum(const float* __restrict__ img, float* run, int W, int H,
                                                         float inv, double* rows) {
  __shared__ double sh[kThreads];
  for (int y = blockIdx.x; y < H; y += gridDim.x) {
    double m[3] = {0.0, 0.0, 0.0};
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
      const size_t p = (size_t)y * W + x;
      for (int c = 0; c < 3; ++c) {
        const float rs = run[3 * p + c] + img[3 * p + c];
        run[3 * p + c] = rs;
        m[c] += (double)(rs * inv);
      }
    }
    for (int c = 0; c < 3; ++c) {
      const double s = block_reduce(m[c], sh);
      if (threadIdx.x == 0) rows[(size_t)y * kSlotsPerRow + c] = s;
    }
  }
}

// totals over rows (in row order per thread, then a fixed tree)
__global__ void __launch_bounds__(kThreads) k_rows_total(int H, int slot, double* rows) {
  __shared__ double sh[kThreads];
  double a = 0.0;
  for (int y = threadIdx.x; y < H; y += blockDim.x) a += rows[(size_t)y * kSlotsPerRow + slot];
  const double s = block_reduce(a, sh);
  if (threadIdx.x == 0) rows[(size_t)kMaxRows * kSlotsPerRow + slot] = s;
}

// pixel estimate (3x3 box of the running mean, floored) and the V_I row sums
__global__ void __launch_bounds__(kThreads) k_rows_estimate(const float* __restrict__ img,
                                                            const float* __restrict__ run, float* est, int W, int H,
                                                            float inv, float outlier, double* rows) {
  __shared__ double sh[kThreads];
  const double npix = (double)W * (double)H;
  const double* tot = rows + (size_t)kMaxRows * kSlotsPerRow;
  const float fl[3] = {1e-3f * (float)(tot[0] / npix), 1e-3f * (float)(tot[1] / npix),
                       1e-3f * (float)(tot[2] / npix)};
  for (int y = blockIdx.x; y < H; y += gridDim.x) {
    double vi = 0.0;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
      const size_t p = (size_t)y * W + x;
      float s[3] = {0.f, 0.f, 0.f};
      int k = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x + dx, yy = y + dy;
          if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
          const size_t q = (size_t)yy * W + xx;
          for (int c = 0; c < 3; ++c) s[c] += run[3 * q + c] * inv;
          ++k;
        }
      for (int c = 0; c < 3; ++c) {
        const float e = fmaxf(fmaxf(s[c] / (float)k, fl[c]), 1e-8f);
        est[3 * p + c] = e;
        const float r = (fminf(img[3 * p + c], outlier * e) - e) / e;
        vi += (double)(r * r);
      }
    }
    const double sv = block_reduce(vi, sh);
    if (threadIdx.x == 0) rows[(size_t)y * kSlotsPerRow + 3] = sv;
  }
}

__global__ void __launch_bounds__(kThreads) k_rows_final(int H, double npix, double rays, double* rows,
                                                         double* out) {
  __shared__ double sh[kThreads];
  double a = 0.0;
  for (int y = threadIdx.x; y < H; y += blockDim.x) a += rows[(size_t)y * kSlotsPerRow + 3];
  const double s = block_reduce(a, sh);
  if (threadIdx.x == 0) {
    out[0] = s / (3.0 * npix);
    out[1] = rays / npix;
  }
}

}  // namespace

extern "C" mars_status mars_image_stats_static(const float* image_rgb, float* run_sum_rgb, float* estimate_rgb,
                                               int32_t width, int32_t height, int32_t n_prev, float outlier,
                                               double rays, double* vi_ci, void* stream) {
  if (!image_rgb || !run_sum_rgb || !estimate_rgb || !vi_ci)
    return mars::set_error(MARS_ERR_INVALID_ARG, "null image, running sum, estimate or V_I/C_I pointer");
  if (width < 1 || height < 1 || (int64_t)width * height > 0x7fffffffll)
    return mars::set_error(MARS_ERR_INVALID_ARG, "bad resolution %d x %d", width, height);
  if (height > kMaxRows)
    return mars::set_error(MARS_ERR_INVALID_ARG,
                           "image height %d exceeds the %d rows of the static scratch of mars_image_stats_static",
                           height, kMaxRows);
  if (n_prev < 0 || !(outlier > 0.0f) || !(rays >= 0.0))
    return mars::set_error(MARS_ERR_INVALID_ARG, "negative n_prev or rays, or non-positive outlier");
  double* rows = nullptr;
  const mars_status s = scratch_address(&rows);
  if (s != MARS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const float inv = 1.0f / (float)(n_prev + 1);
  const int grid = height < 1024 ? height : 1024;
  k_rows_accum<<<grid, kThreads, 0, st>>>(image_rgb, run_sum_rgb, width, height, inv, rows);
  for (int c = 0; c < 3; ++c) k_rows_total<<<1, kThreads, 0, st>>>(height, c, rows);
  k_rows_estimate<<<grid, kThreads, 0, st>>>(image_rgb, run_sum_rgb, estimate_rgb, width, height, inv, outlier,
                                             rows);
  k_rows_final<<<1, kThreads, 0, st>>>(height, (double)width * (double)height, rays, rows, vi_ci);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mars::set_error(MARS_ERR_CUDA, "image statistics launch: %s", cudaGetErrorString(e));
  return MARS_OK;
}
