// lt_static.cu -- lt_frame_mass_static: the per-frame mass reduction of
// lt_render_tiles (sum of pixel values times the pixel area, FP64, fixed
// order) for images the caller already holds, with no device allocation.
//
// Its scratch (the per-block partial sums) is one file-scope device array
// per GPU; the host looks up its address once per device. Every partial is
// written before it is read, so nothing in the scratch has to start at zero.
#include <mutex>

#include "lt.h"
#include "lt_internal.h"

namespace lt {

constexpr int kStaticMaxFrames = 128;  // frames per call
constexpr int kStaticBlocks = 152;     // partial sums per frame (one block per SM of a GB300)
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

// 128 x 152 doubles = 155,648 bytes per device.
static __device__ __align__(256) double g_mass_partials[kStaticMaxFrames * kStaticBlocks];

__device__ __forceinline__ double block_sum(double s, double* ws) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  double w = 0.0;
  if (threadIdx.x < 32) {
    w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
  }
  return w;  // valid in thread 0
}

// Pass 1: block b of frame f sums its contiguous chunk of the frame's pixels.
__global__ void __launch_bounds__(kStaticThreads) k_mass_partials(const float* __restrict__ image, long long npix,
                                                                  double* __restrict__ partials) {
  __shared__ double ws[32];
  const int f = blockIdx.y, b = blockIdx.x;
  const long long chunk = (npix + kStaticBlocks - 1) / kStaticBlocks;
  const long long p0 = (long long)b * chunk;
  const long long p1 = min(npix, p0 + chunk);
  const float* img = image + (long long)f * npix;
  double s = 0.0;
  for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) s += (double)img[p];
  const double w = block_sum(s, ws);
  if (threadIdx.x == 0) partials[f * kStaticBlocks + b] = w;
}

// Pass 2: frame f's partials in block order, times the pixel area.
__global__ void __launch_bounds__(kStaticThreads) k_mass_finish(const double* __restrict__ partials,
                                                                double pixel_area, double* __restrict__ d_mass) {
  __shared__ double ws[32];
  const int f = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < kStaticBlocks; b += blockDim.x) s += partials[f * kStaticBlocks + b];
  const double w = block_sum(s, ws);
  if (threadIdx.x == 0) d_mass[f] = w * pixel_area;
}

// Device address of the scratch, looked up once per device (with that
// device current) and kept for the life of the process.
static lt_status static_scratch(double** out) {
  static std::mutex mu;
  static double* addr[kMaxDevices] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LT_ERR_ARG;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || !p) return LT_ERR_CUDA;
    addr[dev] = static_cast<double*>(p);
  }
  *out = addr[dev];
  return LT_OK;
}

}  // namespace lt

extern "C" lt_status lt_frame_mass_static(const float* d_image, int n_frames, int W, int H, double pixel_area,
                                          double* d_mass, lt_stream stream) {
  if (!d_image || !d_mass || n_frames < 1 || W < 1 || H < 1) return LT_ERR_ARG;
  if (!(pixel_area > 0.0) || !(pixel_area < 1e300)) return LT_ERR_ARG;
  if (n_frames > lt::kStaticMaxFrames) return LT_ERR_CAPACITY;
  double* partials = nullptr;
  const lt_status st = lt::static_scratch(&partials);
  if (st != LT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const long long npix = (long long)W * (long long)H;
  lt::k_mass_partials<<<dim3(lt::kStaticBlocks, n_frames), lt::kStaticThreads, 0, s>>>(d_image, npix, partials);
  if (cudaGetLastError() != cudaSuccess) return LT_ERR_CUDA;
  lt::k_mass_finish<<<n_frames, lt::kStaticThreads, 0, s>>>(partials, pixel_area, d_mass);
  if (cudaGetLastError() != cudaSuccess) return LT_ERR_CUDA;
  return LT_OK;
}
