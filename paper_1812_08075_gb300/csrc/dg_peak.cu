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

// Tensor-core probes: each warp issues `iters` rounds of four independent mma.sync
// accumulations. kind 0: FP64 m8n8k4 (A, B, C, D double; 512 flops per warp-instruction);
// kind 1: TF32 m16n8k8 with FP32 accumulation (2048 flops per warp-instruction).
__global__ void __launch_bounds__(256) k_mma_probe_f64(double *out, int iters) {
  double a = 1e-3 * (threadIdx.x + 1), b = 0.999;
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) { c[i][0] = 1e-3 * i; c[i][1] = 2e-3 * i; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_mma_probe_tf32(float *out, int iters) {
  const unsigned a = __float_as_uint(1e-3f * (threadIdx.x + 1)), b = __float_as_uint(0.999f);
  float c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = 1e-3f * (i + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %4, %4, %4}, {%5, %5}, "
          "{%0, %1, %2, %3};\n"
          : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
          : "r"(a), "r"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Mixed probe: per iteration each warp issues four DMMA (2048 flops) and every thread
// eight DFMA chains (8 x 2 x 32 = 512 flops per warp). Whether the two share one pipe
// shows in the total rate: near the DFMA-only rate if they do, above it if not.
__global__ void __launch_bounds__(256) k_mma_probe_mixed(double *out, int iters) {
  double a = 1e-3 * (threadIdx.x + 1), b = 0.999;
  double c[4][2], f[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) { c[i][0] = 1e-3 * i; c[i][1] = 2e-3 * i; }
#pragma unroll
  for (int i = 0; i < 8; ++i) f[i] = 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = fma(f[i], b, 1e-3);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
#pragma unroll
  for (int i = 0; i < 8; ++i) s += f[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, typename K>
cudaError_t probe_mma(K kern, double flops_per_warp_iter, cudaStream_t s, double *tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0)) != cudaSuccess) return e;
  const int blocks = sms * std::max(per_sm, 1);
  T *out = nullptr;
  if ((e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T))) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 256;
  double best = 0.0;
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    kern<<<blocks, 256, 0, s>>>(out, iters);
    cudaEventRecord(e1, s);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = flops_per_warp_iter * (double)iters * blocks * (256 / 32);
    if (rep >= 2) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    if (rep < 2 && ms > 0.f) iters = (int)std::min(2.0e9, std::max(256.0, iters * (50.0 / ms)));
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = best;
  return e;
}

}  // namespace

extern "C" dg_status dg_measure_mma_peak(int kind, void *stream, double *tflops) {
  if (!tflops || kind < 0 || kind > 2) return dg_record_error(DG_ERR_INVALID_ARG);
  cudaError_t e;
  if (kind == 0)
    e = probe_mma<double>(k_mma_probe_f64, 4 * 512.0, (cudaStream_t)stream, tflops);
  else if (kind == 1)
    e = probe_mma<float>(k_mma_probe_tf32, 4 * 2048.0, (cudaStream_t)stream, tflops);
  else
    e = probe_mma<double>(k_mma_probe_mixed, 4 * 512.0 + 8 * 2 * 32.0, (cudaStream_t)stream, tflops);
  if (e == cudaErrorMemoryAllocation) return dg_record_error(DG_ERR_OOM);
  return e == cudaSuccess ? DG_OK : dg_record_error(DG_ERR_CUDA);
}

extern "C" dg_status dg_measure_fma_peak(int precision, void *stream, double *tflops) {
  if (!tflops || (precision != DG_FP64 && precision != DG_FP32)) return dg_record_error(DG_ERR_INVALID_ARG);
  const cudaError_t e = precision == DG_FP64 ? probe<double>((cudaStream_t)stream, tflops)
                                             : probe<float>((cudaStream_t)stream, tflops);
  if (e == cudaErrorMemoryAllocation) return dg_record_error(DG_ERR_OOM);
  return e == cudaSuccess ? DG_OK : dg_record_error(DG_ERR_CUDA);
}
