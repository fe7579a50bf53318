// Scalar SIPG apply kernels (Eq. diffreac_weak without data terms), templated on the
// number of basis points P = k+1 and Gauss points M per direction.
//
// One apply is three launches on the caller's stream:
//   k_cell  - Algorithm 1 Parts 1-3 for the volume term of each cell, with the 1D
//             contractions of Eq. lowcomplex done axis by axis on cell data staged in
//             shared memory: interpolate the GLL coefficients to the Gauss points
//             (3 sweeps with A^(i)), differentiate there (3 sweeps with the collocated
//             derivative matrix), apply the pointwise volume term, contract with the
//             transposed derivative matrix into a Gauss-point residual R_vol. It also
//             writes, for each of the cell's six faces, the trace u and the reference
//             normal derivative of u at the face Gauss points (facet sum factorisation
//             with m_d = 1 in the normal direction, Sec. 2.2).
//   k_face  - one thread per face quadrature point: jump, average flux and penalty of
//             Eq. diffreac_weak from the two sides' traces, tangential derivatives by the
//             collocated matrix on curved faces, and the face residual of each side as a
//             (value, normal-derivative) pair at the face points. No atomics: every face
//             side is written by exactly one face.
//   k_back  - adds the six face residuals to R_vol along the normal direction and applies
//             the transposed interpolation (A^(i),T, Algorithm 1 Part 3) to produce y.
#pragma once
#include <type_traits>

#include "dg_df64.cuh"
#include "dg_internal.h"

namespace dgk {

template <int P, int M, typename T>
struct SmemTables {
  T interp[M * P];
  T dcol[M * M];
  T e0[M], e1[M], d0[M], d1[M];
  T w[M];
};

template <int P, int M, typename T>
__device__ __forceinline__ void load_tables(SmemTables<P, M, T> &s, const DevTables<T> *g) {
  for (int i = threadIdx.x; i < M * P; i += blockDim.x) s.interp[i] = g->interp[i];
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) s.dcol[i] = g->dcol[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    s.e0[i] = g->e0[i]; s.e1[i] = g->e1[i];
    s.d0[i] = g->d0[i]; s.d1[i] = g->d1[i];
    s.w[i] = g->w[i];
  }
}

template <typename T>
__host__ __device__ constexpr size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

// Issues the copy of n contiguous values of T global -> shared with all of a thread's
// copies in flight at once (cp.async; 16-byte pieces when both ends and the size allow).
// The caller then waits (dg_cp_async_wait_all) and synchronises the block.
template <typename T>
__device__ __forceinline__ void stage_async(T *dst, const T *src, int n, int tid, int nt) {
  constexpr int V = int(16 / sizeof(T));
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && n % V == 0) {
    for (int i = tid; i < n / V; i += nt) dg_cp_async16(dst + i * V, src + i * V);
  } else {
    for (int i = tid; i < n; i += nt) dg_cp_async(dst + i, src + i);
  }
}

// ------------------------------------------------------------------------------------
// k_cell
// ------------------------------------------------------------------------------------
template <int P, int M, typename T>
__host__ __device__ constexpr size_t cell_smem_bytes(int cpb) {
  return align16<T>(sizeof(SmemTables<P, M, T>)) + size_t(4) * cpb * M * M * M * sizeof(T);
}

template <int P, int M, typename T, int GEO, bool KAPPA>
__global__ void __launch_bounds__(256) k_cell(const ScalarArgs<T> a, const io_t<T> *__restrict__ x,
                                              T *__restrict__ rvol, T *__restrict__ traces,
                                              int cpb, int64_t sx, int64_t sr, int64_t st) {
  constexpr int P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<SmemTables<P, M, T> *>(smem_raw);
  T *S0 = reinterpret_cast<T *>(smem_raw + align16<T>(sizeof(SmemTables<P, M, T>)));
  T *S1 = S0 + cpb * M3;
  T *S2 = S1 + cpb * M3;
  T *S3 = S2 + cpb * M3;
  const int tid = threadIdx.x, nt = blockDim.x;
  x += blockIdx.y * sx;
  rvol += blockIdx.y * sr;
  traces += blockIdx.y * st;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  load_tables(tb, a.tab);
  {
    const io_t<T> *xb = x + c0 * P3;
    for (int i = tid; i < nc * P3; i += nt) S0[i] = io_in<T>(xb[i]);
  }
  __syncthreads();
  // axis 0: [c][j2][j1][j0] (P3) -> [c][j2][j1][q0]
  for (int i = tid; i < nc * P * P * M; i += nt) {
    const int c = i / (P * P * M), r = i - c * (P * P * M);
    const int q0 = r % M, j12 = r / M;
    const T *src = S0 + c * P3 + j12 * P;
    Acc<T> acc;
    acc.init(tb.interp[q0 * P], src[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) acc.add(tb.interp[q0 * P + j], src[j]);
    S1[i] = acc.get();
  }
  __syncthreads();
  // axis 1: [c][j2][j1][q0] -> [c][j2][q1][q0]
  for (int i = tid; i < nc * P * M2; i += nt) {
    const int c = i / (P * M2), r = i - c * (P * M2);
    const int q0 = r % M, q1 = (r / M) % M, j2 = r / M2;
    const T *src = S1 + c * (P * P * M) + j2 * (P * M) + q0;
    Acc<T> acc;
    acc.init(tb.interp[q1 * P], src[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) acc.add(tb.interp[q1 * P + j], src[j * M]);
    S0[i] = acc.get();
  }
  __syncthreads();
  // axis 2: [c][j2][q1][q0] -> U = [c][q2][q1][q0]
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, r = i - c * M3;
    const int q01 = r % M2, q2 = r / M2;
    const T *src = S0 + c * (P * M2) + q01;
    Acc<T> acc;
    acc.init(tb.interp[q2 * P], src[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) acc.add(tb.interp[q2 * P + j], src[j * M2]);
    S2[i] = acc.get();
  }
  __syncthreads();
  const T *U = S2;
  // face traces: u and d_n u (reference) at the M^2 points of each of the 6 faces
  {
    T *tr = traces + c0 * (12 * M2);
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
      Acc<T> acc;
      acc.init(row[0], src[0]);
#pragma unroll
      for (int j = 1; j < M; ++j) acc.add(row[j], src[j * stride]);
      tr[i] = acc.get();
    }
  }
  // reference gradient at the Gauss points and the pointwise volume flux
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, q = i - c * M3;
    const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
    const T *u = U + c * M3;
    Acc<T> a0, a1, a2;
    a0.init(tb.dcol[q0 * M], u[q1 * M + q2 * M2]);
    a1.init(tb.dcol[q1 * M], u[q0 + q2 * M2]);
    a2.init(tb.dcol[q2 * M], u[q0 + q1 * M]);
#pragma unroll
    for (int r = 1; r < M; ++r) {
      a0.add(tb.dcol[q0 * M + r], u[r + q1 * M + q2 * M2]);
      a1.add(tb.dcol[q1 * M + r], u[q0 + r * M + q2 * M2]);
      a2.add(tb.dcol[q2 * M + r], u[q0 + q1 * M + r * M2]);
    }
    T g0 = a0.get(), g1 = a1.get(), g2 = a2.get();
    T f0, f1, f2;
    if (GEO == GEO_AFFINE) {
      T W = tb.w[q0] * tb.w[q1] * tb.w[q2];
      if (KAPPA) W *= io_in<T>(a.kappa_vol[(c0 + c) * M3 + q]);
      f0 = (W * a.vol_g[0]) * g0;
      f1 = (W * a.vol_g[1]) * g1;
      f2 = (W * a.vol_g[2]) * g2;
    } else {
      const T *G = a.gvol + (c0 + c) * (7 * M3) + q;
      if (KAPPA) {
        const T kq = io_in<T>(a.kappa_vol[(c0 + c) * M3 + q]);
        g0 *= kq; g1 *= kq; g2 *= kq;
      }
      const T G00 = G[0], G01 = G[M3], G02 = G[2 * M3], G11 = G[3 * M3], G12 = G[4 * M3], G22 = G[5 * M3];
      Acc<T> b0, b1, b2;  // G g, summed from the last term as the nested FMAs would
      b0.init(G02, g2); b0.add(G01, g1); b0.add(G00, g0);
      b1.init(G12, g2); b1.add(G11, g1); b1.add(G01, g0);
      b2.init(G22, g2); b2.add(G12, g1); b2.add(G02, g0);
      f0 = b0.get(); f1 = b1.get(); f2 = b2.get();
    }
    S0[i] = f0;
    S1[i] = f1;
    S3[i] = f2;
  }
  __syncthreads();
  // R_vol = mass * U + D^T f (each direction's transposed derivative along its own axis)
  {
    T *rv = rvol + c0 * M3;
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
      T mw;
      if (GEO == GEO_AFFINE) mw = (tb.w[q0] * tb.w[q1] * tb.w[q2]) * a.vol_m;
      else mw = a.gvol[(c0 + c) * (7 * M3) + 6 * M3 + q];
      Acc<T> acc;
      acc.init(mw, U[i]);
      const T *F0 = S0 + c * M3, *F1 = S1 + c * M3, *F2 = S3 + c * M3;
#pragma unroll
      for (int r = 0; r < M; ++r) {
        acc.add(tb.dcol[r * M + q0], F0[r + q1 * M + q2 * M2]);
        acc.add(tb.dcol[r * M + q1], F1[q0 + r * M + q2 * M2]);
        acc.add(tb.dcol[r * M + q2], F2[q0 + q1 * M + r * M2]);
      }
      rv[i] = acc.get();
    }
  }
}

// ------------------------------------------------------------------------------------
// k_face
// ------------------------------------------------------------------------------------
struct FaceId {
  int axis, t1, t2;
  int64_t cm, cp;  // -1 where absent
};

template <typename T>
__device__ __forceinline__ FaceId decode_face(const ScalarArgs<T> &a, int64_t f) {
  FaceId r;
  const int ax = (f >= a.face_off[1]) + (f >= a.face_off[2]);
  r.axis = ax;
  r.t1 = (ax == 0) ? 1 : 0;
  r.t2 = (ax == 2) ? 1 : 2;
  const int64_t fl = f - (ax == 0 ? a.face_off[0] : (ax == 1 ? a.face_off[1] : a.face_off[2]));
  const int na = ax == 0 ? a.nx : (ax == 1 ? a.ny : a.nz);
  const int n1 = ax == 0 ? a.ny : a.nx;
  const int fa = (int)(fl % (na + 1));
  const int64_t rest = fl / (na + 1);
  const int i1 = (int)(rest % n1);
  const int i2 = (int)(rest / n1);
  // cell coordinates with the axis coordinate set to fa (plus side); minus side is fa-1
  int cx, cy, cz;
  if (ax == 0) { cx = fa; cy = i1; cz = i2; }
  else if (ax == 1) { cx = i1; cy = fa; cz = i2; }
  else { cx = i1; cy = i2; cz = fa; }
  const int64_t cplus = cx + (int64_t)a.nx * (cy + (int64_t)a.ny * cz);
  const int64_t step = ax == 0 ? 1 : (ax == 1 ? (int64_t)a.nx : (int64_t)a.nx * a.ny);
  r.cp = (fa < na) ? cplus : -1;
  r.cm = (fa > 0) ? cplus - step : -1;
  return r;
}

// The FP32 and double-float face kernels on curved faces copy their faces' traces and
// stored geometry into shared memory with asynchronous copies (all of a thread's loads in
// flight at once). The FP64 kernels, bound by their FP64 arithmetic, load them directly:
// asynchronous staging measured within +-3 % for them at Q2-Q5.
template <typename T>
__host__ __device__ constexpr bool face_async_stage() {
  return !std::is_same<T, double>::value;
}

template <int M, typename T>
__host__ __device__ constexpr size_t face_smem_bytes(int fpb, int geo) {
  return align16<T>(sizeof(SmemTables<1, M, T>)) + align16<T>(fpb * sizeof(FaceId)) +
         (geo == GEO_AFFINE ? 0 : size_t(face_async_stage<T>() ? 16 : 9) * fpb * M * M * sizeof(T));
}

// trace / face-residual addressing: [cell][lf][qty][M^2]
template <int M>
__device__ __forceinline__ int64_t tr_idx(int64_t cell, int lf, int qty, int qf) {
  return ((cell * 6 + lf) * 2 + qty) * (M * M) + qf;
}

template <int M, typename T, int GEO, bool KAPPA>
__global__ void __launch_bounds__(256) k_face(const ScalarArgs<T> a, const T *__restrict__ traces,
                                              T *__restrict__ fres, int fpb, int64_t st) {
  constexpr int M2 = M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<SmemTables<1, M, T> *>(smem_raw);
  // the block's faces, decoded once (64-bit divisions) and read by every point
  FaceId *sF = reinterpret_cast<FaceId *>(smem_raw + align16<T>(sizeof(SmemTables<1, M, T>)));
  T *SM = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(sF) + align16<T>(fpb * sizeof(FaceId)));
  const int tid = threadIdx.x, nt = blockDim.x;
  traces += blockIdx.y * st;
  fres += blockIdx.y * st;
  const int64_t f0 = (int64_t)blockIdx.x * fpb;
  const int nf = (int)min((int64_t)fpb, a.nface - f0);
  for (int i = tid; i < nf; i += nt) sF[i] = decode_face(a, f0 + i);
  // tables: only the weights are needed here (dcol on curved faces)
  for (int i = tid; i < M * M; i += nt) tb.dcol[i] = a.tab->dcol[i];
  for (int i = tid; i < M; i += nt) tb.w[i] = a.tab->w[i];
  __syncthreads();
  const T sc = a.sc, ss = a.ss, half = T(0.5);
  if (GEO == GEO_AFFINE) {
    for (int i = tid; i < nf * M2; i += nt) {
      const int lfc = i / M2, qf = i - lfc * M2;
      const FaceId &F = sF[lfc];
      const int ax = F.axis;
      const int qs = qf % M, qt = qf / M;
      const T W = tb.w[qs] * tb.w[qt];
      const T bW = W * a.face_b[ax], pw = W * a.face_pw[ax];
      if (F.cm >= 0 && F.cp >= 0) {
        const T um = traces[tr_idx<M>(F.cm, 2 * ax + 1, 0, qf)];
        const T dm = traces[tr_idx<M>(F.cm, 2 * ax + 1, 1, qf)];
        const T up = traces[tr_idx<M>(F.cp, 2 * ax, 0, qf)];
        const T dp = traces[tr_idx<M>(F.cp, 2 * ax, 1, qf)];
        T km = T(1), kp = T(1);
        if (KAPPA) {
          km = io_in<T>(a.kappa_face[(F.cm * 6 + 2 * ax + 1) * M2 + qf]);
          kp = io_in<T>(a.kappa_face[(F.cp * 6 + 2 * ax) * M2 + qf]);
        }
        const T J = um - up;
        const T flux = half * bW * fma(km, dm, kp * dp);
        const T Rv = fma(sc, flux, pw * J);
        const T sJ = ss * half * J * bW;
        fres[tr_idx<M>(F.cm, 2 * ax + 1, 0, qf)] = Rv;
        fres[tr_idx<M>(F.cm, 2 * ax + 1, 1, qf)] = KAPPA ? sJ * km : sJ;
        fres[tr_idx<M>(F.cp, 2 * ax, 0, qf)] = -Rv;
        fres[tr_idx<M>(F.cp, 2 * ax, 1, qf)] = KAPPA ? sJ * kp : sJ;
      } else {
        const int side = F.cm >= 0 ? 1 : 0;
        const int64_t cb = side ? F.cm : F.cp;
        const int lf = 2 * ax + side;
        T Rv = T(0), Rn = T(0);
        if ((a.dmask >> lf) & 1u) {
          const T u = traces[tr_idx<M>(cb, lf, 0, qf)];
          const T d = traces[tr_idx<M>(cb, lf, 1, qf)];
          const T kb = KAPPA ? io_in<T>(a.kappa_face[(cb * 6 + lf) * M2 + qf]) : T(1);
          const T b = side ? bW : -bW;  // outward normal
          Rv = fma(sc * kb, b * d, pw * u);
          Rn = ss * kb * u * b;
        }
        fres[tr_idx<M>(cb, lf, 0, qf)] = Rv;
        fres[tr_idx<M>(cb, lf, 1, qf)] = Rn;
      }
    }
    return;
  }
  // curved faces (stored geometry): stage traces, pointwise terms, tangential back-projection
  constexpr bool ASYNC = face_async_stage<T>();
  T *sU = SM;                   // [face][4][M2]: u-, dn-, u+, dn+
  T *sR = SM + 4 * fpb * M2;    // [face][5][M2]: Rv, Rt1-, Rt2-, Rt1+, Rt2+
  T *sG = SM + 9 * fpb * M2;    // [face][7][M2]: the faces' stored geometry (ASYNC)
  if constexpr (ASYNC) {
    // a face's trace row (M^2 values) and the block's geometry in 16-byte pieces where their
    // sizes allow (every start is then 16-byte aligned), else one value at a time
    constexpr int V = (M2 * sizeof(T)) % 16 == 0 ? int(16 / sizeof(T)) : 1;
    for (int i = tid; i < nf * 4 * (M2 / V); i += nt) {
      const int lfc = i / (4 * (M2 / V)), r = i - lfc * (4 * (M2 / V));
      const int slot = r / (M2 / V), qf = (r - slot * (M2 / V)) * V;
      const FaceId &F = sF[lfc];
      const int ax = F.axis;
      const T *src = nullptr;
      if (slot < 2) {
        if (F.cm >= 0) src = traces + tr_idx<M>(F.cm, 2 * ax + 1, slot, qf);
        else src = traces + tr_idx<M>(F.cp, 2 * ax, slot, qf);  // boundary face at the lower end
      } else if (F.cm >= 0 && F.cp >= 0) {
        src = traces + tr_idx<M>(F.cp, 2 * ax, slot - 2, qf);
      }
      T *dst = sU + lfc * (4 * M2) + slot * M2 + qf;
      if constexpr (V > 1) {
        if (src) dg_cp_async16(dst, src);
        else *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        if (src) dg_cp_async(dst, src);
        else *dst = T(0);
      }
    }
    // the block's faces are consecutive: their geometry is one contiguous range
    const T *g0 = a.gface + f0 * (7 * M2);
    if constexpr (V > 1) {
      for (int i = tid; i < nf * 7 * (M2 / V); i += nt) dg_cp_async16(sG + i * V, g0 + i * V);
    } else {
      for (int i = tid; i < nf * 7 * M2; i += nt) dg_cp_async(sG + i, g0 + i);
    }
    dg_cp_async_wait_all();
  } else {
    for (int i = tid; i < nf * 4 * M2; i += nt) {
      const int lfc = i / (4 * M2), r = i - lfc * (4 * M2);
      const int slot = r / M2, qf = r - slot * M2;
      const FaceId &F = sF[lfc];
      const int ax = F.axis;
      T v = T(0);
      if (slot < 2) {
        if (F.cm >= 0) v = traces[tr_idx<M>(F.cm, 2 * ax + 1, slot, qf)];
        else v = traces[tr_idx<M>(F.cp, 2 * ax, slot, qf)];  // boundary face at the lower end
      } else if (F.cm >= 0 && F.cp >= 0) {
        v = traces[tr_idx<M>(F.cp, 2 * ax, slot - 2, qf)];
      }
      sU[i] = v;
    }
  }
  __syncthreads();
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const int64_t f = f0 + lfc;
    const FaceId &F = sF[lfc];
    const int ax = F.axis, t1 = F.t1, t2 = F.t2;
    const int qs = qf % M, qt = qf / M;
    const T *gf = ASYNC ? sG + lfc * (7 * M2) + qf : a.gface + f * (7 * M2) + qf;
    const T *u0 = sU + lfc * 4 * M2;
    T *R = sR + lfc * 5 * M2;
    // tangential reference derivatives of side "-" (slot 0) or the single boundary side
    Acc<T> d1, d2;
    d1.init(tb.dcol[qs * M], u0[qt * M]);
    d2.init(tb.dcol[qt * M], u0[qs]);
#pragma unroll
    for (int r = 1; r < M; ++r) {
      d1.add(tb.dcol[qs * M + r], u0[r + qt * M]);
      d2.add(tb.dcol[qt * M + r], u0[qs + r * M]);
    }
    const T ds1 = d1.get(), ds2 = d2.get();
    // the face's geometry vector in the normal and the two tangential directions, picked by
    // selects (indexing a local array with the run-time axes would put it in local memory)
    const T g0 = gf[0], g1 = gf[M2], g2 = gf[2 * M2];
    const T bmn = dg_pick3(g0, g1, g2, ax), bm1 = dg_pick3(g0, g1, g2, t1), bm2 = dg_pick3(g0, g1, g2, t2);
    Acc<T> gacc;
    gacc.init(bm2, ds2); gacc.add(bm1, ds1); gacc.add(bmn, u0[M2 + qf]);
    const T gm = gacc.get();
    const T pw = gf[6 * M2];
    if (F.cm >= 0 && F.cp >= 0) {
      const T *u1 = u0 + 2 * M2;
      Acc<T> e1, e2;
      e1.init(tb.dcol[qs * M], u1[qt * M]);
      e2.init(tb.dcol[qt * M], u1[qs]);
#pragma unroll
      for (int r = 1; r < M; ++r) {
        e1.add(tb.dcol[qs * M + r], u1[r + qt * M]);
        e2.add(tb.dcol[qt * M + r], u1[qs + r * M]);
      }
      const T es1 = e1.get(), es2 = e2.get();
      const T h0 = gf[3 * M2], h1 = gf[4 * M2], h2 = gf[5 * M2];
      const T bpn = dg_pick3(h0, h1, h2, ax), bp1 = dg_pick3(h0, h1, h2, t1), bp2 = dg_pick3(h0, h1, h2, t2);
      Acc<T> pacc;
      pacc.init(bp2, es2); pacc.add(bp1, es1); pacc.add(bpn, u1[M2 + qf]);
      const T gp = pacc.get();
      T km = T(1), kp = T(1);
      if (KAPPA) {
        km = io_in<T>(a.kappa_face[(F.cm * 6 + 2 * ax + 1) * M2 + qf]);
        kp = io_in<T>(a.kappa_face[(F.cp * 6 + 2 * ax) * M2 + qf]);
      }
      const T J = u0[qf] - u1[qf];
      const T flux = half * fma(km, gm, kp * gp);
      const T Rv = fma(sc, flux, pw * J);
      const T sJ = ss * half * J;
      const T sm = KAPPA ? sJ * km : sJ, sp = KAPPA ? sJ * kp : sJ;
      R[qf] = Rv;
      R[M2 + qf] = sm * bm1;
      R[2 * M2 + qf] = sm * bm2;
      R[3 * M2 + qf] = sp * bp1;
      R[4 * M2 + qf] = sp * bp2;
      fres[tr_idx<M>(F.cm, 2 * ax + 1, 1, qf)] = sm * bmn;
      fres[tr_idx<M>(F.cp, 2 * ax, 1, qf)] = sp * bpn;
    } else {
      const int side = F.cm >= 0 ? 1 : 0;
      const int64_t cb = side ? F.cm : F.cp;
      const int lf = 2 * ax + side;
      T Rv = T(0), s1 = T(0), s2 = T(0), sn = T(0);
      if ((a.dmask >> lf) & 1u) {
        const T kb = KAPPA ? io_in<T>(a.kappa_face[(cb * 6 + lf) * M2 + qf]) : T(1);
        const T u = u0[qf];
        Rv = fma(sc * kb, gm, pw * u);
        const T su = ss * kb * u;
        s1 = su * bm1;
        s2 = su * bm2;
        sn = su * bmn;
      }
      R[qf] = Rv;
      R[M2 + qf] = s1;
      R[2 * M2 + qf] = s2;
      fres[tr_idx<M>(cb, lf, 1, qf)] = sn;
    }
  }
  __syncthreads();
  // value residual of each side: Rv + dcol^T (tangential terms)
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const FaceId &F = sF[lfc];
    const int ax = F.axis;
    const int qs = qf % M, qt = qf / M;
    const T *R = sR + lfc * 5 * M2;
    Acc<T> vm;
    vm.set(R[qf]);
#pragma unroll
    for (int r = 0; r < M; ++r) {
      vm.add(tb.dcol[r * M + qs], R[M2 + r + qt * M]);
      vm.add(tb.dcol[r * M + qt], R[2 * M2 + qs + r * M]);
    }
    if (F.cm >= 0 && F.cp >= 0) {
      Acc<T> vp;
      vp.set(-R[qf]);
#pragma unroll
      for (int r = 0; r < M; ++r) {
        vp.add(tb.dcol[r * M + qs], R[3 * M2 + r + qt * M]);
        vp.add(tb.dcol[r * M + qt], R[4 * M2 + qs + r * M]);
      }
      fres[tr_idx<M>(F.cm, 2 * ax + 1, 0, qf)] = vm.get();
      fres[tr_idx<M>(F.cp, 2 * ax, 0, qf)] = vp.get();
    } else {
      const int side = F.cm >= 0 ? 1 : 0;
      fres[tr_idx<M>(side ? F.cm : F.cp, 2 * ax + side, 0, qf)] = vm.get();
    }
  }
}

// ------------------------------------------------------------------------------------
// k_back
// ------------------------------------------------------------------------------------
template <int P, int M, typename T>
__host__ __device__ constexpr size_t back_smem_bytes(int cpb) {
  return align16<T>(sizeof(SmemTables<P, M, T>)) + size_t(cpb) * (2 * M * M * M + 12 * M * M) * sizeof(T);
}

template <int P, int M, typename T>
__global__ void __launch_bounds__(256) k_back(const ScalarArgs<T> a, const T *__restrict__ rvol,
                                              const T *__restrict__ fres, io_t<T> *__restrict__ y, int cpb,
                                              int64_t sy, int64_t sr, int64_t st) {
  constexpr int P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<SmemTables<P, M, T> *>(smem_raw);
  T *S0 = reinterpret_cast<T *>(smem_raw + align16<T>(sizeof(SmemTables<P, M, T>)));
  T *S1 = S0 + cpb * M3;
  T *SF = S1 + cpb * M3;
  const int tid = threadIdx.x, nt = blockDim.x;
  y += blockIdx.y * sy;
  rvol += blockIdx.y * sr;
  fres += blockIdx.y * st;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  load_tables(tb, a.tab);
  for (int i = tid; i < nc * M3; i += nt) S0[i] = rvol[c0 * M3 + i];
  for (int i = tid; i < nc * 12 * M2; i += nt) SF[i] = fres[c0 * 12 * M2 + i];
  __syncthreads();
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, q = i - c * M3;
    const int qv[3] = {q % M, (q / M) % M, q / M2};
    const T *sf = SF + c * 12 * M2;
    Acc<T> acc;
    acc.set(S0[i]);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int qa = qv[ax];
      const int qf = (ax == 0) ? qv[1] + M * qv[2] : (ax == 1 ? qv[0] + M * qv[2] : qv[0] + M * qv[1]);
      const T *lo = sf + (2 * ax) * 2 * M2, *hi = sf + (2 * ax + 1) * 2 * M2;
      acc.add(tb.e0[qa], lo[qf]);
      acc.add(tb.d0[qa], lo[M2 + qf]);
      acc.add(tb.e1[qa], hi[qf]);
      acc.add(tb.d1[qa], hi[M2 + qf]);
    }
    S1[i] = acc.get();
  }
  __syncthreads();
  // transposed interpolation, axis 0: [c][q2][q1][q0] -> [c][q2][q1][j0]
  for (int i = tid; i < nc * M2 * P; i += nt) {
    const int c = i / (M2 * P), r = i - c * (M2 * P);
    const int j0 = r % P, q12 = r / P;
    const T *src = S1 + c * M3 + q12 * M;
    Acc<T> acc;
    acc.init(tb.interp[j0], src[0]);
#pragma unroll
    for (int q = 1; q < M; ++q) acc.add(tb.interp[q * P + j0], src[q]);
    S0[i] = acc.get();
  }
  __syncthreads();
  // axis 1: [c][q2][q1][j0] -> [c][q2][j1][j0]
  for (int i = tid; i < nc * M * P * P; i += nt) {
    const int c = i / (M * P * P), r = i - c * (M * P * P);
    const int j0 = r % P, j1 = (r / P) % P, q2 = r / (P * P);
    const T *src = S0 + c * (M2 * P) + q2 * (M * P) + j0;
    Acc<T> acc;
    acc.init(tb.interp[j1], src[0]);
#pragma unroll
    for (int q = 1; q < M; ++q) acc.add(tb.interp[q * P + j1], src[q * P]);
    S1[i] = acc.get();
  }
  __syncthreads();
  // axis 2: [c][q2][j1][j0] -> y [c][j2][j1][j0]
  {
    io_t<T> *yb = y + c0 * P3;
    for (int i = tid; i < nc * P3; i += nt) {
      const int c = i / P3, r = i - c * P3;
      const int j01 = r % (P * P), j2 = r / (P * P);
      const T *src = S1 + c * (M * P * P) + j01;
      Acc<T> acc;
      acc.init(tb.interp[j2], src[0]);
#pragma unroll
      for (int q = 1; q < M; ++q) acc.add(tb.interp[q * P + j2], src[q * P * P]);
      yb[i] = io_out(acc.get());
    }
  }
}

}  // namespace dgk
