// DG Stokes block operator of Eq. (stokes_weak) (Sec. 5.3) on affine (axis-parallel
// unit-cube lattice) meshes: velocity u in (Q_k)^3, pressure p in Q_{k-1}, viscous SIPG
// block on each component, -(p, div v) - (div u, q) in the volume and
// ({p}, [v].n) + ([u].n, {q}) on interior and Dirichlet faces.
//
// Same three phases as the scalar apply. k_stokes_cell interpolates the pressure and,
// component by component, the velocity to the Gauss points (Eq. lowcomplex), writes the
// face traces, forms the viscous flux with the pressure term on the diagonal and
// accumulates the divergence; k_stokes_face adds the coupling terms to the component
// normal to the face (on axis-parallel faces n = +-e_a, Sec. 5.3's simplification of
// grad u n to d_a u); k_stokes_back lifts the face residuals and contracts back with the
// transposed velocity and pressure interpolation matrices.
#include "dg_scalar_kernels.cuh"

namespace dgs {

using dgk::align16;
using dgk::decode_face;
using dgk::FaceId;

template <int P, int M, typename T>
struct Tabs {
  T interp[M * P];
  T interp_p[M * (P - 1)];
  T dcol[M * M];
  T e0[M], e1[M], d0[M], d1[M];
  T w[M];
};

template <int P, int M, typename T>
__device__ __forceinline__ void load_tabs(Tabs<P, M, T> &s, const DevTables<T> *g) {
  for (int i = threadIdx.x; i < M * P; i += blockDim.x) s.interp[i] = g->interp[i];
  for (int i = threadIdx.x; i < M * (P - 1); i += blockDim.x) s.interp_p[i] = g->interp_p[i];
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) s.dcol[i] = g->dcol[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    s.e0[i] = g->e0[i]; s.e1[i] = g->e1[i];
    s.d0[i] = g->d0[i]; s.d1[i] = g->d1[i];
    s.w[i] = g->w[i];
  }
}

// 1D contractions of a block of cells along one axis. Extents of the input per cell:
// (A0, A1, A2) with axis 0 fastest; the contracted axis has N input and O output points.
// Coefficient of output o and input n: mat[o*N + n], or mat[n*O + o] when TR (transposed).
template <int N, int O, int A1, int A2, bool TR, typename T>
__device__ __forceinline__ void contract0(const T *in, int ics, T *out, int ocs, const T *mat, int nc) {
  for (int i = threadIdx.x; i < nc * O * A1 * A2; i += blockDim.x) {
    const int c = i / (O * A1 * A2), r = i - c * (O * A1 * A2);
    const int o = r % O, k12 = r / O;
    const T *src = in + c * ics + k12 * N;
    Acc<T> acc;
    acc.init(TR ? mat[o] : mat[o * N], src[0]);
#pragma unroll
    for (int n = 1; n < N; ++n) acc.add(TR ? mat[n * O + o] : mat[o * N + n], src[n]);
    out[c * ocs + r] = acc.get();
  }
}

template <int A0, int N, int O, int A2, bool TR, typename T>
__device__ __forceinline__ void contract1(const T *in, int ics, T *out, int ocs, const T *mat, int nc) {
  for (int i = threadIdx.x; i < nc * A0 * O * A2; i += blockDim.x) {
    const int c = i / (A0 * O * A2), r = i - c * (A0 * O * A2);
    const int k0 = r % A0, o = (r / A0) % O, k2 = r / (A0 * O);
    const T *src = in + c * ics + k2 * (N * A0) + k0;
    Acc<T> acc;
    acc.init(TR ? mat[o] : mat[o * N], src[0]);
#pragma unroll
    for (int n = 1; n < N; ++n) acc.add(TR ? mat[n * O + o] : mat[o * N + n], src[n * A0]);
    out[c * ocs + r] = acc.get();
  }
}

// (the output may be the FP64 result vector of a double-float apply: TO = io_t<T>)
template <int A01, int N, int O, bool TR, typename T, typename TO>
__device__ __forceinline__ void contract2(const T *in, int ics, TO *out, int ocs, const T *mat, int nc) {
  for (int i = threadIdx.x; i < nc * A01 * O; i += blockDim.x) {
    const int c = i / (A01 * O), r = i - c * (A01 * O);
    const int k01 = r % A01, o = r / A01;
    const T *src = in + c * ics + k01;
    Acc<T> acc;
    acc.init(TR ? mat[o] : mat[o * N], src[0]);
#pragma unroll
    for (int n = 1; n < N; ++n) acc.add(TR ? mat[n * O + o] : mat[o * N + n], src[n * A01]);
    store_to(out + c * ocs + r, acc.get());
  }
}

// values at the Gauss points from Q_{NI-1} coefficients: in [c][NI^3] -> out [c][M^3]
template <int NI, int M, typename T>
__device__ __forceinline__ void to_gauss(const T *in, int ics, T *t1, T *t2, T *out, const T *mat, int nc) {
  contract0<NI, M, NI, NI, false>(in, ics, t1, M * NI * NI, mat, nc);
  __syncthreads();
  contract1<M, NI, M, NI, false>(t1, M * NI * NI, t2, M * M * NI, mat, nc);
  __syncthreads();
  contract2<M * M, NI, M, false>(t2, M * M * NI, out, M * M * M, mat, nc);
  __syncthreads();
}

// transposed: Gauss-point residual [c][M^3] -> coefficients out (global, stride ocs)
template <int NO, int M, typename T, typename TO>
__device__ __forceinline__ void from_gauss(const T *in, T *t1, T *t2, TO *out, int ocs, const T *mat, int nc) {
  contract0<M, NO, M, M, true>(in, M * M * M, t1, NO * M * M, mat, nc);
  __syncthreads();
  contract1<NO, M, NO, M, true>(t1, NO * M * M, t2, NO * NO * M, mat, nc);
  __syncthreads();
  contract2<NO * NO, M, NO, true>(t2, NO * NO * M, out, ocs, mat, nc);
}

constexpr int kTr = 42;  // trace / face-residual slots per cell: 3 x (6 faces x 2) + 6 pressure

template <int P, typename T>
__host__ __device__ constexpr size_t cell_smem(int cpb) {
  return align16<T>(sizeof(Tabs<P, P, T>)) +
         (size_t(cpb) * (3 * P * P * P + (P - 1) * (P - 1) * (P - 1) + 8 * P * P * P) + 4 * P * P * P) * sizeof(T);
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_stokes_cell(const ScalarArgs<T> a, const T mu, const io_t<T> *__restrict__ x,
                                                     T *__restrict__ rvol, T *__restrict__ traces, int cpb,
                                                     int64_t sx, int64_t sr, int64_t st) {
  constexpr int M = P, PP = P - 1, P3 = P * P * P, PP3 = PP * PP * PP, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<Tabs<P, M, T> *>(smem_raw);
  T *Xu = reinterpret_cast<T *>(smem_raw + align16<T>(sizeof(Tabs<P, M, T>)));
  T *Xp = Xu + cpb * 3 * P3;
  T *T1 = Xp + cpb * PP3, *T2 = T1 + cpb * M3, *PG = T2 + cpb * M3, *U = PG + cpb * M3;
  T *F = U + cpb * M3, *DV = F + 3 * cpb * M3;
  T *WG = DV + cpb * M3;  // per point: W mu G_dd (3) and W detJ, shared by the block's cells
  const int tid = threadIdx.x, nt = blockDim.x;
  x += blockIdx.y * sx;
  rvol += blockIdx.y * sr;
  traces += blockIdx.y * st;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  load_tabs(tb, a.tab);
  for (int i = tid; i < nc * 3 * P3; i += nt) Xu[i] = io_in<T>(x[c0 * 3 * P3 + i]);
  for (int i = tid; i < nc * PP3; i += nt) Xp[i] = io_in<T>(x[a.ncell * 3 * P3 + c0 * PP3 + i]);
  for (int i = tid; i < nc * M3; i += nt) DV[i] = T(0);
  const T hinv[3] = {T(a.nx), T(a.ny), T(a.nz)};
  const T V = a.vol;
  __syncthreads();  // tables loaded
  for (int q = tid; q < M3; q += nt) {
    const T W = tb.w[q % M] * tb.w[(q / M) % M] * tb.w[q / M2];
    WG[q] = W * mu * a.vol_g[0];
    WG[M3 + q] = W * mu * a.vol_g[1];
    WG[2 * M3 + q] = W * mu * a.vol_g[2];
    WG[3 * M3 + q] = W * V;
  }
  __syncthreads();
  to_gauss<PP, M>(Xp, PP3, T1, T2, PG, tb.interp_p, nc);
  for (int comp = 0; comp < 3; ++comp) {
    to_gauss<P, M>(Xu + comp * P3, 3 * P3, T1, T2, U, tb.interp, nc);
    T *tr = traces + c0 * (kTr * M2);
    for (int i = tid; i < nc * 12 * M2; i += nt) {
      const int c = i / (12 * M2), r = i - c * (12 * M2);
      const int lq = r / M2, qf = r - lq * M2;
      const int lf = lq >> 1, qty = lq & 1, ax = lf >> 1, side = lf & 1;
      const int qs = qf % M, qt = qf / M;
      int base, stride;
      if (ax == 0) { base = M * (qs + M * qt); stride = 1; }
      else if (ax == 1) { base = qs + M2 * qt; stride = M; }
      else { base = qs + M * qt; stride = M2; }
      const T *row = side ? (qty ? tb.d1 : tb.e1) : (qty ? tb.d0 : tb.e0);
      const T *src = U + c * M3 + base;
      T acc = row[0] * src[0];
#pragma unroll
      for (int j = 1; j < M; ++j) acc = fma(row[j], src[j * stride], acc);
      tr[c * (kTr * M2) + comp * 12 * M2 + r] = acc;
    }
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
      const T *u = U + c * M3;
      T g0 = tb.dcol[q0 * M] * u[q1 * M + q2 * M2];
      T g1 = tb.dcol[q1 * M] * u[q0 + q2 * M2];
      T g2 = tb.dcol[q2 * M] * u[q0 + q1 * M];
#pragma unroll
      for (int r = 1; r < M; ++r) {
        g0 = fma(tb.dcol[q0 * M + r], u[r + q1 * M + q2 * M2], g0);
        g1 = fma(tb.dcol[q1 * M + r], u[q0 + r * M + q2 * M2], g1);
        g2 = fma(tb.dcol[q2 * M + r], u[q0 + q1 * M + r * M2], g2);
      }
      T f[3] = {WG[q] * g0, WG[M3 + q] * g1, WG[2 * M3 + q] * g2};
      const T gd = comp == 0 ? g0 : (comp == 1 ? g1 : g2);
      // -(p, d_comp v_comp): coefficient of the reference derivative d_comp is -W V/h p
      f[comp] = fma(-WG[3 * M3 + q] * hinv[comp], PG[i], f[comp]);
      DV[i] = fma(hinv[comp], gd, DV[i]);
      F[i] = f[0];
      F[cpb * M3 + i] = f[1];
      F[2 * cpb * M3 + i] = f[2];
    }
    __syncthreads();
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
      const T *F0 = F + c * M3, *F1 = F + cpb * M3 + c * M3, *F2 = F + 2 * cpb * M3 + c * M3;
      T acc = tb.dcol[q0] * F0[q1 * M + q2 * M2];
      acc = fma(tb.dcol[q1], F1[q0 + q2 * M2], acc);
      acc = fma(tb.dcol[q2], F2[q0 + q1 * M], acc);
#pragma unroll
      for (int r = 1; r < M; ++r) {
        acc = fma(tb.dcol[r * M + q0], F0[r + q1 * M + q2 * M2], acc);
        acc = fma(tb.dcol[r * M + q1], F1[q0 + r * M + q2 * M2], acc);
        acc = fma(tb.dcol[r * M + q2], F2[q0 + q1 * M + r * M2], acc);
      }
      rvol[(c0 + c) * 4 * M3 + comp * M3 + q] = acc;
    }
    __syncthreads();
  }
  // pressure: traces (values) and the Gauss-point residual of -(div u, q)
  {
    T *tr = traces + c0 * (kTr * M2);
    for (int i = tid; i < nc * 6 * M2; i += nt) {
      const int c = i / (6 * M2), r = i - c * (6 * M2);
      const int lf = r / M2, qf = r - lf * M2;
      const int ax = lf >> 1, side = lf & 1;
      const int qs = qf % M, qt = qf / M;
      int base, stride;
      if (ax == 0) { base = M * (qs + M * qt); stride = 1; }
      else if (ax == 1) { base = qs + M2 * qt; stride = M; }
      else { base = qs + M * qt; stride = M2; }
      const T *row = side ? tb.e1 : tb.e0;
      const T *src = PG + c * M3 + base;
      T acc = row[0] * src[0];
#pragma unroll
      for (int j = 1; j < M; ++j) acc = fma(row[j], src[j * stride], acc);
      tr[c * (kTr * M2) + 36 * M2 + r] = acc;
    }
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
      const T W = tb.w[q0] * tb.w[q1] * tb.w[q2];
      rvol[(c0 + c) * 4 * M3 + 3 * M3 + q] = -(W * V) * DV[i];
    }
  }
}

template <int M, typename T>
__global__ void __launch_bounds__(256) k_stokes_face(const ScalarArgs<T> a, const T mu,
                                                     const T *__restrict__ traces, T *__restrict__ fres, int fpb,
                                                     int64_t st) {
  constexpr int M2 = M * M;
  __shared__ T sw[M];
  const int tid = threadIdx.x, nt = blockDim.x;
  traces += blockIdx.y * st;
  fres += blockIdx.y * st;
  for (int i = tid; i < M; i += nt) sw[i] = a.tab->w[i];
  __syncthreads();
  const int64_t f0 = (int64_t)blockIdx.x * fpb;
  const int nf = (int)min((int64_t)fpb, a.nface - f0);
  const T sc = a.sc, ss = a.ss, half = T(0.5);
  auto TR = [&](int64_t cell, int slot, int qf) -> int64_t { return (cell * kTr + slot) * M2 + qf; };
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const FaceId F = decode_face(a, f0 + lfc);
    const int ax = F.axis;
    const int qs = qf % M, qt = qf / M;
    const T W = sw[qs] * sw[qt];
    const T bW = W * a.face_b[ax], pw = W * a.face_pw[ax], wds = W * a.face_area[ax];
    if (F.cm >= 0 && F.cp >= 0) {
      const int lm = 2 * ax + 1, lp = 2 * ax;
      const T pavg = half * (traces[TR(F.cm, 36 + lm, qf)] + traces[TR(F.cp, 36 + lp, qf)]);
      T jn = T(0);
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const T um = traces[TR(F.cm, comp * 12 + 2 * lm, qf)], dm = traces[TR(F.cm, comp * 12 + 2 * lm + 1, qf)];
        const T up = traces[TR(F.cp, comp * 12 + 2 * lp, qf)], dp = traces[TR(F.cp, comp * 12 + 2 * lp + 1, qf)];
        const T J = um - up;
        const T flux = half * mu * bW * (dm + dp);
        T Rv = fma(sc, flux, pw * J);
        if (comp == ax) { Rv = fma(wds, pavg, Rv); jn = J; }
        const T sJ = ss * half * mu * J * bW;
        fres[TR(F.cm, comp * 12 + 2 * lm, qf)] = Rv;
        fres[TR(F.cm, comp * 12 + 2 * lm + 1, qf)] = sJ;
        fres[TR(F.cp, comp * 12 + 2 * lp, qf)] = -Rv;
        fres[TR(F.cp, comp * 12 + 2 * lp + 1, qf)] = sJ;
      }
      const T Rq = half * wds * jn;
      fres[TR(F.cm, 36 + lm, qf)] = Rq;
      fres[TR(F.cp, 36 + lp, qf)] = Rq;
    } else {
      const int side = F.cm >= 0 ? 1 : 0;
      const int64_t cb = side ? F.cm : F.cp;
      const int lf = 2 * ax + side;
      const bool dir = (a.dmask >> lf) & 1u;
      const T nrm = side ? T(1) : T(-1);
      const T b = nrm * bW;
      T Rq = T(0);
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        T Rv = T(0), Rn = T(0);
        if (dir) {
          const T u = traces[TR(cb, comp * 12 + 2 * lf, qf)], d = traces[TR(cb, comp * 12 + 2 * lf + 1, qf)];
          Rv = fma(sc * mu, b * d, pw * u);
          Rn = ss * mu * u * b;
          if (comp == ax) {
            Rv = fma(wds * nrm, traces[TR(cb, 36 + lf, qf)], Rv);
            Rq = wds * nrm * u;
          }
        }
        fres[TR(cb, comp * 12 + 2 * lf, qf)] = Rv;
        fres[TR(cb, comp * 12 + 2 * lf + 1, qf)] = Rn;
      }
      fres[TR(cb, 36 + lf, qf)] = Rq;
    }
  }
}

template <int P, typename T>
__host__ __device__ constexpr size_t back_smem(int cpb) {
  return align16<T>(sizeof(Tabs<P, P, T>)) + size_t(cpb) * (3 * P * P * P + kTr * P * P) * sizeof(T);
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_stokes_back(const ScalarArgs<T> a, const T *__restrict__ rvol,
                                                     const T *__restrict__ fres, io_t<T> *__restrict__ y, int cpb,
                                                     int64_t sy, int64_t sr, int64_t st) {
  constexpr int M = P, PP = P - 1, P3 = P * P * P, PP3 = PP * PP * PP, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<Tabs<P, M, T> *>(smem_raw);
  T *R = reinterpret_cast<T *>(smem_raw + align16<T>(sizeof(Tabs<P, M, T>)));
  T *T1 = R + cpb * M3, *T2 = T1 + cpb * M3, *SF = T2 + cpb * M3;
  const int tid = threadIdx.x, nt = blockDim.x;
  y += blockIdx.y * sy;
  rvol += blockIdx.y * sr;
  fres += blockIdx.y * st;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  load_tabs(tb, a.tab);
  for (int i = tid; i < nc * kTr * M2; i += nt) SF[i] = fres[c0 * kTr * M2 + i];
  for (int comp = 0; comp < 4; ++comp) {
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      R[i] = rvol[(c0 + c) * 4 * M3 + comp * M3 + q];
    }
    __syncthreads();
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int qv[3] = {q % M, (q / M) % M, q / M2};
      const T *sf = SF + c * kTr * M2;
      Acc<T> acc;
      acc.set(R[i]);
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int qa = qv[ax];
        const int qf = (ax == 0) ? qv[1] + M * qv[2] : (ax == 1 ? qv[0] + M * qv[2] : qv[0] + M * qv[1]);
        if (comp < 3) {
          const T *lo = sf + (comp * 12 + 4 * ax) * M2, *hi = lo + 2 * M2;
          acc.add(tb.e0[qa], lo[qf]);
          acc.add(tb.d0[qa], lo[M2 + qf]);
          acc.add(tb.e1[qa], hi[qf]);
          acc.add(tb.d1[qa], hi[M2 + qf]);
        } else {
          acc.add(tb.e0[qa], sf[(36 + 2 * ax) * M2 + qf]);
          acc.add(tb.e1[qa], sf[(36 + 2 * ax + 1) * M2 + qf]);
        }
      }
      T1[i] = acc.get();
    }
    __syncthreads();
    if (comp < 3) {
      // y_u[c][comp]: contract T1 -> coefficients, through T2 and R as scratch
      from_gauss<P, M>(T1, T2, R, y + c0 * 3 * P3 + comp * P3, 3 * P3, tb.interp, nc);
    } else {
      from_gauss<PP, M>(T1, T2, R, y + a.ncell * 3 * P3 + c0 * PP3, PP3, tb.interp_p, nc);
    }
    __syncthreads();
  }
}

inline int threads_for(int work) {
  int t = ((work + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

template <int P, typename T>
cudaError_t apply_p(const ScalarArgs<T> &a, T mu, const io_t<T> *x, io_t<T> *y, T *rvol, T *tr, T *fres, int nrhs, int64_t sdof,
                    int64_t srv, int64_t str, int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev) {
  constexpr int M = P, M2 = M * M, M3 = M * M * M;
  cudaError_t e;
  {
    size_t sm = cell_smem<P, T>(cpb);
    auto k = k_stokes_cell<P, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    k<<<dim3((unsigned)((a.ncell + cpb - 1) / cpb), nrhs), threads_for(cpb * M3), sm, s>>>(a, mu, x, rvol, tr, cpb,
                                                                                              sdof, srv, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    if (ev) cudaEventRecord(ev[1], s);
    k_stokes_face<M, T><<<dim3((unsigned)((a.nface + fpb - 1) / fpb), nrhs), threads_for(fpb * M2), 0, s>>>(
        a, mu, tr, fres, fpb, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    size_t sm = back_smem<P, T>(cpb);
    auto k = k_stokes_back<P, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], s);
    k<<<dim3((unsigned)((a.ncell + cpb - 1) / cpb), nrhs), threads_for(cpb * M3), sm, s>>>(a, rvol, fres, y, cpb, sdof,
                                                                                              srv, str);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], s);
  }
  return cudaSuccess;
}

}  // namespace dgs

template <typename T>
cudaError_t launch_stokes_apply(int p, const ScalarArgs<T> &a, T mu, const io_t<T> *x, io_t<T> *y, T *rvol, T *traces, T *fres,
                                int nrhs, int64_t sdof, int64_t srv, int64_t str, int cpb, int fpb, cudaStream_t s,
                                const cudaEvent_t *ev) {
  switch (p) {
    case 3: return dgs::apply_p<3, T>(a, mu, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
    case 4: return dgs::apply_p<4, T>(a, mu, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
    case 5: return dgs::apply_p<5, T>(a, mu, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
    case 6: return dgs::apply_p<6, T>(a, mu, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_stokes_apply<double>(int, const ScalarArgs<double> &, double, const double *, double *,
                                                 double *, double *, double *, int, int64_t, int64_t, int64_t, int,
                                                 int, cudaStream_t, const cudaEvent_t *);
template cudaError_t launch_stokes_apply<float>(int, const ScalarArgs<float> &, float, const float *, float *, float *,
                                                float *, float *, int, int64_t, int64_t, int64_t, int, int,
                                                cudaStream_t, const cudaEvent_t *);
template cudaError_t launch_stokes_apply<df64>(int, const ScalarArgs<df64> &, df64, const double *, double *, df64 *,
                                               df64 *, df64 *, int, int64_t, int64_t, int64_t, int, int, cudaStream_t,
                                               const cudaEvent_t *);
