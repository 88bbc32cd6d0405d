// Internal helpers shared by the CUDA translation units of the XL-BOMD library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <atomic>
#include <cstdint>
#include <cstddef>

namespace xl {

// Number of kernels this library has launched (all contexts, all streams).
extern std::atomic<long long> g_launch_count;
extern thread_local long long t_launch_count;   // launches by the calling host thread
inline void note_launch() {
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  ++t_launch_count;
}

constexpr int kMaxRank = 8;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 doubles */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

}  // namespace xl
