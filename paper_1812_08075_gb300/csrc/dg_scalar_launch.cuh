// Launchers of the scalar apply kernels; included by one translation unit per precision.
#pragma once
#include "dg_scalar_kernels.cuh"

namespace dgk {

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

inline int threads_for(int work) {
  int t = ((work + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}

template <int P, int M, typename T, int GEO, bool KAPPA>
static cudaError_t apply_pmk(const ScalarArgs<T> &a, const T *x, T *y, T *rvol, T *traces, T *fres,
                             int nrhs, int64_t sdof, int64_t srv, int64_t str, int cpb, int fpb,
                             cudaStream_t s, const cudaEvent_t *ev) {
  constexpr int M2 = M * M, M3 = M * M * M;
  cudaError_t e;
  {
    size_t sm = cell_smem_bytes<P, M, T>(cpb);
    auto k = k_cell<P, M, T, GEO, KAPPA>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((unsigned)((a.ncell + cpb - 1) / cpb), nrhs);
    if (ev) cudaEventRecord(ev[0], s);
    k<<<grid, threads_for(cpb * M3), sm, s>>>(a, x, rvol, traces, cpb, sdof, srv, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    size_t sm = face_smem_bytes<M, T>(fpb, GEO == GEO_AFFINE ? GEO_AFFINE : GEO_STORED);
    auto k = k_face<M, T, GEO, KAPPA>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((unsigned)((a.nface + fpb - 1) / fpb), nrhs);
    if (ev) cudaEventRecord(ev[1], s);
    k<<<grid, threads_for(fpb * M2), sm, s>>>(a, traces, fres, fpb, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    size_t sm = back_smem_bytes<P, M, T>(cpb);
    auto k = k_back<P, M, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((unsigned)((a.ncell + cpb - 1) / cpb), nrhs);
    if (ev) cudaEventRecord(ev[2], s);
    k<<<grid, threads_for(cpb * M3), sm, s>>>(a, rvol, fres, y, cpb, sdof, srv, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], s);
  }
  return cudaSuccess;
}

template <int P, int M, typename T>
static cudaError_t apply_p(int geo, bool kappa, const ScalarArgs<T> &a, const T *x, T *y, T *rvol,
                           T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str,
                           int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev) {
  if (geo == GEO_AFFINE) {
    if (kappa) return apply_pmk<P, M, T, GEO_AFFINE, true>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
    return apply_pmk<P, M, T, GEO_AFFINE, false>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
  }
  if (geo == GEO_STORED) {
    if (kappa) return apply_pmk<P, M, T, GEO_STORED, true>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
    return apply_pmk<P, M, T, GEO_STORED, false>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dgk

template <typename T>
cudaError_t launch_scalar_apply(int p, int m, int geo, bool kappa, const ScalarArgs<T> &a, const T *x, T *y,
                                T *rvol, T *traces, T *fres, int nrhs, int64_t stride_dofs,
                                int64_t stride_rvol, int64_t stride_tr, int cpb, int fpb, cudaStream_t s,
                                const cudaEvent_t *ev) {
#define DGK_CASE(PP, MM)                                                                                      \
  if (p == PP && m == MM)                                                                                     \
    return dgk::apply_p<PP, MM, T>(geo, kappa, a, x, y, rvol, traces, fres, nrhs, stride_dofs, stride_rvol, \
                                   stride_tr, cpb, fpb, s, ev);
  DGK_CASE(2, 2) DGK_CASE(3, 3) DGK_CASE(4, 4) DGK_CASE(5, 5) DGK_CASE(6, 6)
  DGK_CASE(2, 3) DGK_CASE(3, 4) DGK_CASE(4, 5) DGK_CASE(5, 6) DGK_CASE(6, 7)
#undef DGK_CASE
  return cudaErrorInvalidValue;
}
