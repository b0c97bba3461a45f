// Arithmetic-pipe ceilings of the GPU the library runs on, measured by throughput loops: the
// FP64 fused multiply-add (the pipe that bounds the IEEE FP64 hopping term), the scalar FP32
// FMA and the packed FP32x2 FMA (the pipes of the FP32 / FP16 / BF16 kernels). Each thread runs
// independent FMA chains long enough that the loop, not the launch, sets the time; the result
// is flops per second over the whole device (2 flops per FMA, 4 per packed FMA).
#include <cuda_runtime.h>

#include "../../include/grid_dwf.h"

namespace {

constexpr int PEAK_CHAINS = 8;    // independent accumulators per thread (hide the FMA latency)
constexpr int PEAK_ITERS = 4096;  // loop trips per thread
constexpr int PEAK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_loop(T a, T b, T* sink, int flag) {
  T v[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) v[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < PEAK_ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += v[c];
  if (flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // flag is 0 at run time: keeps the loop live
}

__global__ void __launch_bounds__(PEAK_THREADS) k_ffma2_loop(float a, float b, float* sink, int flag) {
  float2 v[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) v[c] = make_float2((float)threadIdx.x + c, (float)c);
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  for (int i = 0; i < PEAK_ITERS; ++i) {
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) v[c] = __ffma2_rn(v[c], A, B);
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += v[c].x + v[c].y;
  if (flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int grid_dwf_pipe_peak(int kind, void* stream, double* gflops) {
  if (!gflops || kind < GRID_DWF_PEAK_FP64_FMA || kind > GRID_DWF_PEAK_FP32X2_FMA) return GRID_DWF_ERR_INVALID_ARG;
  *gflops = 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GRID_DWF_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = sms * 8;  // 8 resident CTAs of 256 threads per SM
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GRID_DWF_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GRID_DWF_ERR_CUDA;
  }
  double best = 0;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // rep 0 warms up
    cudaEventRecord(e0, st);
    switch (kind) {
      case GRID_DWF_PEAK_FP64_FMA: k_fma_loop<double><<<blocks, PEAK_THREADS, 0, st>>>(1.0000001, 1e-9, nullptr, 0); break;
      case GRID_DWF_PEAK_FP32_FMA: k_fma_loop<float><<<blocks, PEAK_THREADS, 0, st>>>(1.0001f, 1e-6f, nullptr, 0); break;
      default: k_ffma2_loop<<<blocks, PEAK_THREADS, 0, st>>>(1.0001f, 1e-6f, nullptr, 0); break;
    }
    cudaEventRecord(e1, st);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && ms > 0) {
      const double flops_per_fma = kind == GRID_DWF_PEAK_FP32X2_FMA ? 4.0 : 2.0;
      const double flops = (double)blocks * PEAK_THREADS * PEAK_ITERS * PEAK_CHAINS * flops_per_fma;
      const double g = flops / (ms * 1e-3) / 1e9;
      if (g > best) best = g;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return GRID_DWF_ERR_CUDA;
  *gflops = best;
  return GRID_DWF_OK;
}
