// Double-float instantiation of the scalar apply kernels (DG_VARIANT_DF64) and the
// conversion of FP64 tables and geometry to double-float.
#include "dg_scalar_launch.cuh"

template cudaError_t launch_scalar_apply<df64>(int, int, int, bool, const ScalarArgs<df64> &, const double *, double *,
                                               df64 *, df64 *, df64 *, int, int64_t, int64_t, int64_t, int, int,
                                               cudaStream_t, const cudaEvent_t *, LaunchInfo *, int, int64_t, int64_t,
                                               const HostTables *);

namespace {
__global__ void k_to_df64(const double *__restrict__ in, df64 *__restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = io_in<df64>(in[i]);
}
}  // namespace

cudaError_t convert_to_df64(const double *in, df64 *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  const int64_t cap = 32 * (int64_t)dg_device_sms();
  k_to_df64<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
