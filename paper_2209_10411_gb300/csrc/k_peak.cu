// FMA throughput microbenchmark: the measured FP32 and FP64 ALU peaks that
// the library's ALU-bound kernels (contacts, flagging, shape fitting) are
// reported against.
#include <cuda_runtime.h>

#include "mi_peak.h"

namespace mi {
void set_thread_error(const char* msg);  // engine.cu: message for mi_delbm_last_error(NULL)
}

namespace {
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_UNROLL = 16;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return __fmaf_rn(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return __fma_rn(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T a, T b, int iters, float* __restrict__ out) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u) {
#pragma unroll
      for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fma_t(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

template <typename T>
mi_status run_peak(int iters, double* tflops, double* ms_out, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, 256, 0);
  if (e != cudaSuccess || sms <= 0 || per_sm <= 0) {
    mi::set_thread_error("mi_measure_fma_peak: device query failed");
    return MI_ECUDA;
  }
  const int blocks = sms * per_sm;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * 256 * (size_t)blocks) != cudaSuccess) {
    cudaGetLastError();
    mi::set_thread_error("mi_measure_fma_peak: device allocation failed");
    return MI_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = (T)0.9999999, b = (T)1e-7;
  k_fma_peak<T><<<blocks, 256, 0, s>>>(a, b, iters, out);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_peak<T><<<blocks, 256, 0, s>>>(a, b, iters, out);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) {
    mi::set_thread_error("mi_measure_fma_peak: kernel failed");
    return MI_ECUDA;
  }
  const double flop = 2.0 * PEAK_CHAINS * PEAK_UNROLL * (double)iters * 256.0 * (double)blocks;
  *tflops = flop / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return MI_OK;
}
}  // namespace

extern "C" mi_status mi_measure_fma_peak(int precision, double* tflops_out, double* ms_out, void* stream) {
  if (!tflops_out || (precision != 0 && precision != 1)) {
    mi::set_thread_error("mi_measure_fma_peak: precision must be 0 (FP32) or 1 (FP64), tflops_out non-null");
    return MI_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // about 15 ms at the nominal rates (FP32 ~80 TFLOP/s, FP64 ~1.2 TFLOP/s)
  return precision == 0 ? run_peak<float>(16384, tflops_out, ms_out, s) : run_peak<double>(256, tflops_out, ms_out, s);
}
