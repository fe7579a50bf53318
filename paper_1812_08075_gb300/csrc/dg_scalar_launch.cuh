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

// Fills q with the shape of a launch of kernel k instead of launching it.
template <typename Kern>
static cudaError_t query_launch(Kern k, dim3 grid, int threads, size_t sm, LaunchInfo *q) {
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, threads, sm);
  if (e != cudaSuccess) return e;
  q->blocks = (int64_t)grid.x * grid.y;
  q->threads = threads;
  q->blocks_per_sm = bps;
  q->items = q->blocks;
  return cudaSuccess;
}

template <int P, int M, typename T, int GEO, bool KAPPA>
static cudaError_t apply_pmk(const ScalarArgs<T> &a, const io_t<T> *x, io_t<T> *y, T *rvol, T *traces, T *fres,
                             int nrhs, int64_t sdof, int64_t srv, int64_t str, int cpb, int fpb,
                             cudaStream_t s, const cudaEvent_t *ev, LaunchInfo *q) {
  constexpr int M2 = M * M, M3 = M * M * M;
  cudaError_t e;
  if (q) {
    const dim3 gc((unsigned)((a.ncell + cpb - 1) / cpb), nrhs), gf((unsigned)((a.nface + fpb - 1) / fpb), nrhs);
    const size_t s0 = cell_smem_bytes<P, M, T>(cpb), s2 = back_smem_bytes<P, M, T>(cpb);
    const size_t s1 = face_smem_bytes<M, T>(fpb, GEO == GEO_AFFINE ? GEO_AFFINE : GEO_STORED);
    if ((e = set_smem(k_cell<P, M, T, GEO, KAPPA>, s0)) != cudaSuccess ||
        (e = set_smem(k_face<M, T, GEO, KAPPA>, s1)) != cudaSuccess || (e = set_smem(k_back<P, M, T>, s2)) != cudaSuccess)
      return e;
    if ((e = query_launch(k_cell<P, M, T, GEO, KAPPA>, gc, threads_for(cpb * M3), s0, q)) != cudaSuccess) return e;
    if ((e = query_launch(k_face<M, T, GEO, KAPPA>, gf, threads_for(fpb * M2), s1, q + 1)) != cudaSuccess) return e;
    return query_launch(k_back<P, M, T>, gc, threads_for(cpb * M3), s2, q + 2);
  }
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
static cudaError_t apply_p(int geo, bool kappa, const ScalarArgs<T> &a, const io_t<T> *x, io_t<T> *y, T *rvol,
                           T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str,
                           int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev, LaunchInfo *q) {
  if (geo == GEO_AFFINE) {
    if (kappa) return apply_pmk<P, M, T, GEO_AFFINE, true>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev, q);
    return apply_pmk<P, M, T, GEO_AFFINE, false>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev, q);
  }
  if (geo == GEO_STORED) {
    if (kappa) return apply_pmk<P, M, T, GEO_STORED, true>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev, q);
    return apply_pmk<P, M, T, GEO_STORED, false>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev, q);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dgk

template <typename T>
cudaError_t launch_scalar_apply(int p, int m, int geo, bool kappa, const ScalarArgs<T> &a, const io_t<T> *x, io_t<T> *y,
                                T *rvol, T *traces, T *fres, int nrhs, int64_t stride_dofs,
                                int64_t stride_rvol, int64_t stride_tr, int cpb, int fpb, cudaStream_t s,
                                const cudaEvent_t *ev, LaunchInfo *query) {
#define DGK_CASE(PP, MM)                                                                                      \
  if (p == PP && m == MM)                                                                                     \
    return dgk::apply_p<PP, MM, T>(geo, kappa, a, x, y, rvol, traces, fres, nrhs, stride_dofs, stride_rvol, \
                                   stride_tr, cpb, fpb, s, ev, query);
  DGK_CASE(2, 2) DGK_CASE(3, 3) DGK_CASE(4, 4) DGK_CASE(5, 5) DGK_CASE(6, 6)
  DGK_CASE(2, 3) DGK_CASE(3, 4) DGK_CASE(4, 5) DGK_CASE(5, 6) DGK_CASE(6, 7)
#undef DGK_CASE
  return cudaErrorInvalidValue;
}
