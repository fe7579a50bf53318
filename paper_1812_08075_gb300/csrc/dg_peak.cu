// Throughput probe of the FP64 and FP32 FMA pipes (dg_measure_fma_peak): every thread
// runs eight independent FMA chains, enough warps per SM to hide the FMA latency, so the
// kernel issues FMAs at the pipe's rate. Used by measurement harnesses beside the peak
// derived from the pipe's per-clock rate and the SM clock.
#include <algorithm>

#include "dg_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = a[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) s += a[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t probe(cudaStream_t s, double *tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, 256, 0)) != cudaSuccess) return e;
  const int blocks = sms * std::max(per_sm, 1);
  T *out = nullptr;
  if ((e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T))) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T b = T(0.999), c = T(1e-3);
  // calibrate to about 50 ms per launch, then keep the best of three launches
  int iters = 1024;
  double best = 0.0;
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<blocks, 256, 0, s>>>(out, iters, b, c);
    cudaEventRecord(e1, s);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8.0 * (double)iters * blocks * 256;
    if (rep >= 2) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    if (rep < 2 && ms > 0.f) {
      const double scale = 50.0 / ms;
      iters = (int)std::min(2.0e9, std::max(1024.0, iters * scale));
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = best;
  return e;
}

}  // namespace

extern "C" dg_status dg_measure_fma_peak(int precision, void *stream, double *tflops) {
  if (!tflops || (precision != DG_FP64 && precision != DG_FP32)) return dg_record_error(DG_ERR_INVALID_ARG);
  const cudaError_t e = precision == DG_FP64 ? probe<double>((cudaStream_t)stream, tflops)
                                             : probe<float>((cudaStream_t)stream, tflops);
  if (e == cudaErrorMemoryAllocation) return dg_record_error(DG_ERR_OOM);
  return e == cudaSuccess ? DG_OK : dg_record_error(DG_ERR_CUDA);
}
