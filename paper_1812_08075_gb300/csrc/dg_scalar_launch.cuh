// Launchers of the scalar apply kernels; included by one translation unit per precision.
#pragma once
#include <type_traits>

#include "dg_scalar_lines.cuh"

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

// Cells [cb, cb + cn) of the cell-side kernels as a launch of their own: the arguments with
// every per-cell array offset to cb and ncell = cn.
template <int P, int M, typename T>
static ScalarArgs<T> cell_range(const ScalarArgs<T> &a, int64_t cb, int64_t cn) {
  ScalarArgs<T> r = a;
  r.ncell = cn;
  if (r.gvol) r.gvol += cb * 7 * M * M * M;
  if (r.kappa_vol) r.kappa_vol += cb * M * M * M;
  return r;
}

// phases: bit 0 the cell kernel, bit 1 the face kernel, bit 2 the back-projection kernel;
// the cell-side kernels take cells [cb, cb + cn) (cn < 0: all cells).
template <int P, int M, typename T, int GEO, bool KAPPA>
static cudaError_t apply_pmk(const ScalarArgs<T> &a, const io_t<T> *x, io_t<T> *y, T *rvol, T *traces, T *fres,
                             int nrhs, int64_t sdof, int64_t srv, int64_t str, int cpb, int fpb,
                             cudaStream_t s, const cudaEvent_t *ev, LaunchInfo *q, int phases = 7, int64_t cb = 0,
                             int64_t cn = -1, const HostTables *ht = nullptr) {
  // line-per-thread cell and back kernels for FP32 and double-float (same grid, block and
  // shared memory as the thread-per-point ones); FP64 keeps the thread-per-point kernels
  const bool lines = ht != nullptr && !std::is_same<T, double>::value;
  LineTab<P, M, T> lt;
  if (lines) lt = line_tables<P, M, T>(*ht);
  constexpr int P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  cudaError_t e;
  if (cn < 0) { cb = 0; cn = a.ncell; }
  const ScalarArgs<T> ac = cell_range<P, M, T>(a, cb, cn);
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
  if ((phases & 1) && cn > 0) {
    size_t sm = cell_smem_bytes<P, M, T>(cpb);
    auto k = k_cell<P, M, T, GEO, KAPPA>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((unsigned)((cn + cpb - 1) / cpb), nrhs);
    if (ev) cudaEventRecord(ev[0], s);
    if (lines) {
      auto kl = k_cell_lines<P, M, T, GEO, KAPPA>;
      if ((e = set_smem(kl, sm)) != cudaSuccess) return e;
      kl<<<grid, threads_for(cpb * M3), sm, s>>>(ac, lt, x + cb * P3, rvol + cb * M3, traces + cb * 12 * M2, cpb, sdof,
                                                 srv, str);
    } else {
      k<<<grid, threads_for(cpb * M3), sm, s>>>(ac, x + cb * P3, rvol + cb * M3, traces + cb * 12 * M2, cpb, sdof, srv,
                                                str);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (phases & 2) {
    size_t sm = face_smem_bytes<M, T>(fpb, GEO == GEO_AFFINE ? GEO_AFFINE : GEO_STORED);
    auto k = k_face<M, T, GEO, KAPPA>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((unsigned)((a.nface + fpb - 1) / fpb), nrhs);
    if (ev) cudaEventRecord(ev[1], s);
    k<<<grid, threads_for(fpb * M2), sm, s>>>(a, traces, fres, fpb, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((phases & 4) && cn > 0) {
    size_t sm = back_smem_bytes<P, M, T>(cpb);
    auto k = k_back<P, M, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((unsigned)((cn + cpb - 1) / cpb), nrhs);
    if (ev) cudaEventRecord(ev[2], s);
    if (lines) {
      auto kl = k_back_lines<P, M, T>;
      if ((e = set_smem(kl, sm)) != cudaSuccess) return e;
      kl<<<grid, threads_for(cpb * M3), sm, s>>>(ac, lt, rvol + cb * M3, fres + cb * 12 * M2, y + cb * P3, cpb, sdof,
                                                 srv, str);
    } else {
      k<<<grid, threads_for(cpb * M3), sm, s>>>(ac, rvol + cb * M3, fres + cb * 12 * M2, y + cb * P3, cpb, sdof, srv,
                                                str);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], s);
  }
  return cudaSuccess;
}

template <int P, int M, typename T>
static cudaError_t apply_p(int geo, bool kappa, const ScalarArgs<T> &a, const io_t<T> *x, io_t<T> *y, T *rvol,
                           T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str,
                           int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev, LaunchInfo *q, int ph,
                           int64_t cb, int64_t cn, const HostTables *ht) {
#define DGK_PMK(G, K) \
  return apply_pmk<P, M, T, G, K>(a, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev, q, ph, cb, cn, ht)
  if (geo == GEO_AFFINE) {
    if (kappa) DGK_PMK(GEO_AFFINE, true);
    DGK_PMK(GEO_AFFINE, false);
  }
  if (geo == GEO_STORED) {
    if (kappa) DGK_PMK(GEO_STORED, true);
    DGK_PMK(GEO_STORED, false);
  }
#undef DGK_PMK
  return cudaErrorInvalidValue;
}

}  // namespace dgk

template <typename T>
cudaError_t launch_scalar_apply(int p, int m, int geo, bool kappa, const ScalarArgs<T> &a, const io_t<T> *x, io_t<T> *y,
                                T *rvol, T *traces, T *fres, int nrhs, int64_t stride_dofs,
                                int64_t stride_rvol, int64_t stride_tr, int cpb, int fpb, cudaStream_t s,
                                const cudaEvent_t *ev, LaunchInfo *query, int phases, int64_t cell_begin,
                                int64_t cell_count, const HostTables *ht) {
#define DGK_CASE(PP, MM)                                                                                      \
  if (p == PP && m == MM)                                                                                     \
    return dgk::apply_p<PP, MM, T>(geo, kappa, a, x, y, rvol, traces, fres, nrhs, stride_dofs, stride_rvol, \
                                   stride_tr, cpb, fpb, s, ev, query, phases, cell_begin, cell_count, ht);
  DGK_CASE(2, 2) DGK_CASE(3, 3) DGK_CASE(4, 4) DGK_CASE(5, 5) DGK_CASE(6, 6)
  DGK_CASE(2, 3) DGK_CASE(3, 4) DGK_CASE(4, 5) DGK_CASE(5, 6) DGK_CASE(6, 7)
#undef DGK_CASE
  return cudaErrorInvalidValue;
}
