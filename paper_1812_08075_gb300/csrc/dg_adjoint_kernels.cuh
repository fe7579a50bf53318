// Adjoint of the scalar SIPG operator for L = 0.5 ||A(kappa) x - b||^2 (FP64 or double-float).
//
// Given r = A x - b: y = A^T r, i.e. the bilinear form with trial and test swapped,
// a(v, u) (Eq. diffreac_weak): the same kernels with the face coefficients of the flux
// term -n.{kappa grad u}[v] and the symmetry term theta [u] n.{kappa grad v} exchanged.
// The derivative with respect to each per-point kappa value is r^T (dA/dkappa_q) x:
//   volume:  grad_ref r^T G grad_ref x                          (G = W detJ J^-1 J^-T),
//   faces:   w (-(b.grad_ref x)[r] + theta [x] (b.grad_ref r))   (w = 1/2 interior, 1 Dirichlet),
// with b = W J^-1 n_vec of the side that owns the value. x and r are evaluated together
// (the two-input fusion of Sec. 3.3) and the geometry is recomputed from the vertex
// coordinates in the kernels, so nothing stored per quadrature point is needed.
#pragma once
#include <type_traits>

#include "dg_geo_device.cuh"
#include "dg_scalar_kernels.cuh"

namespace dga {

using namespace dgk;

// dkappa entry: overwritten, or (acc) added to, for the sum over right-hand sides. Each
// entry is written by exactly one thread of a launch, so no atomics are needed.
template <typename T>
__device__ __forceinline__ void put_dk(io_t<T> *p, const T &v, bool acc) {
  if (acc) {
    io_t<T> t;
    store_to(&t, v);
    *p += t;
  } else {
    store_to(p, v);
  }
}

template <int P, int M, typename T>
struct Tab {
  T interp[M * P];
  T dcol[M * M];
  T e0[M], e1[M], d0[M], d1[M];
  T w[M], s[M];
};

template <int P, int M, typename T>
__device__ __forceinline__ void load_tab(Tab<P, M, T> &t, const DevTables<T> *g) {
  for (int i = threadIdx.x; i < M * P; i += blockDim.x) t.interp[i] = g->interp[i];
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) t.dcol[i] = g->dcol[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    t.e0[i] = g->e0[i]; t.e1[i] = g->e1[i]; t.d0[i] = g->d0[i]; t.d1[i] = g->d1[i];
    t.w[i] = g->w[i]; t.s[i] = g->s[i];
  }
}

// Coefficients -> values at the Gauss points for nc cells: x (global, packed P^3 per
// cell) -> U [c][M^3], through scratch buffers A0, A1 (each >= nc M^3).
template <int P, int M, typename T>
__device__ void to_gauss(const io_t<T> *__restrict__ xg, T *A0, T *A1, T *U, const T *interp, int nc) {
  constexpr int P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < nc * P3; i += nt) A0[i] = io_in<T>(xg[i]);
  __syncthreads();
  for (int i = tid; i < nc * P * P * M; i += nt) {
    const int c = i / (P * P * M), r = i - c * (P * P * M);
    const int q0 = r % M, j12 = r / M;
    const T *src = A0 + c * P3 + j12 * P;
    Acc<T> acc;
    acc.init(interp[q0 * P], src[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) acc.add(interp[q0 * P + j], src[j]);
    A1[i] = acc.get();
  }
  __syncthreads();
  for (int i = tid; i < nc * P * M2; i += nt) {
    const int c = i / (P * M2), r = i - c * (P * M2);
    const int q0 = r % M, q1 = (r / M) % M, j2 = r / M2;
    const T *src = A1 + c * (P * P * M) + j2 * (P * M) + q0;
    Acc<T> acc;
    acc.init(interp[q1 * P], src[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) acc.add(interp[q1 * P + j], src[j * M]);
    A0[i] = acc.get();
  }
  __syncthreads();
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, r = i - c * M3;
    const int q01 = r % M2, q2 = r / M2;
    const T *src = A0 + c * (P * M2) + q01;
    Acc<T> acc;
    acc.init(interp[q2 * P], src[0]);
#pragma unroll
    for (int j = 1; j < P; ++j) acc.add(interp[q2 * P + j], src[j * M2]);
    U[i] = acc.get();
  }
  __syncthreads();
}

template <int P, int M, typename T>
__device__ void write_traces(const T *U, T *__restrict__ tr, const Tab<P, M, T> &tb, int nc) {
  constexpr int M2 = M * M, M3 = M * M * M;
  for (int i = threadIdx.x; i < nc * 12 * M2; i += blockDim.x) {
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

template <int P, int M, typename T>
constexpr size_t cell_adj_smem(int cpb) {
  return align16<T>(sizeof(Tab<P, M, T>)) + size_t(cpb) * (8 * M * M * M + 36) * sizeof(T);
}

// nlmode (block-uniform): 0 linear; 1 adds beta (r^3, v) (the residual operator of the
// semilinear reaction); 2 adds 3 beta (x^2 r, v) (its Jacobian action at x, which is then
// evaluated at the Gauss points together with r: the two-input evaluation of Sec. 3).
template <int P, int GEO, bool KAPPA, bool DK, typename T>
__global__ void __launch_bounds__(256) k_cell_adj(const ScalarArgs<T> a, const io_t<T> *__restrict__ r,
                                                  const io_t<T> *__restrict__ x, T *__restrict__ rvol,
                                                  T *__restrict__ tr_r, T *__restrict__ tr_x,
                                                  io_t<T> *__restrict__ dk_vol, int cpb, int nlmode, double beta,
                                                  bool dk_acc) {
  constexpr int M = P, P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<Tab<P, M, T> *>(smem_raw);
  T *A0 = reinterpret_cast<T *>(smem_raw + align16<T>(sizeof(Tab<P, M, T>)));
  T *A1 = A0 + cpb * M3, *Ur = A1 + cpb * M3, *Ux = Ur + cpb * M3;
  T *F0 = Ux + cpb * M3, *F1 = F0 + cpb * M3, *F2 = F1 + cpb * M3, *MW = F2 + cpb * M3;
  T *CC = MW + cpb * M3;  // 36 Jacobian coefficients per cell
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  load_tab(tb, a.tab);
  if (GEO == GEO_RECOMPUTE) {
    for (int c = tid; c < nc; c += nt) {
      double V[8][3], C[3][4][3];
      dgg::cell_corners(a.verts, a.nx, a.ny, c0 + c, V);
      dgg::jacobian_coeffs(V, C);
      for (int k = 0; k < 36; ++k) CC[c * 36 + k] = io_in<T>((&C[0][0][0])[k]);
    }
  }
  const T cT = io_in<T>(a.c), betaT = io_in<T>(beta);
  to_gauss<P, M>(r + c0 * P3, A0, A1, Ur, tb.interp, nc);
  if (DK || nlmode == 2) to_gauss<P, M>(x + c0 * P3, A0, A1, Ux, tb.interp, nc);
  write_traces<P, M>(Ur, tr_r + c0 * 12 * M2, tb, nc);
  if (DK) write_traces<P, M>(Ux, tr_x + c0 * 12 * M2, tb, nc);
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, q = i - c * M3;
    const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
    const T *u = Ur + c * M3;
    Acc<T> a0, a1, a2;
    a0.init(tb.dcol[q0 * M], u[q1 * M + q2 * M2]);
    a1.init(tb.dcol[q1 * M], u[q0 + q2 * M2]);
    a2.init(tb.dcol[q2 * M], u[q0 + q1 * M]);
#pragma unroll
    for (int k = 1; k < M; ++k) {
      a0.add(tb.dcol[q0 * M + k], u[k + q1 * M + q2 * M2]);
      a1.add(tb.dcol[q1 * M + k], u[q0 + k * M + q2 * M2]);
      a2.add(tb.dcol[q2 * M + k], u[q0 + q1 * M + k * M2]);
    }
    const T g0 = a0.get(), g1 = a1.get(), g2 = a2.get();
    const T W = tb.w[q0] * tb.w[q1] * tb.w[q2];
    T G[6], mw, wdet;
    if (GEO == GEO_AFFINE) {
      G[0] = W * a.vol_g[0]; G[1] = T(0); G[2] = T(0); G[3] = W * a.vol_g[1]; G[4] = T(0); G[5] = W * a.vol_g[2];
      mw = W * a.vol_m;
      if constexpr (std::is_same<T, df64>::value) wdet = W * a.vol;
      else wdet = W / T((double)a.nx * a.ny * a.nz);
    } else {
      T J[3][3], A[3][3];
      dgg::jacobian_from_coeffs(CC + c * 36, tb.s[q0], tb.s[q1], tb.s[q2], J);
      const T det = dgg::adjugate(J, A);
      const T sW = W / det;
      int e = 0;
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = rr; cc < 3; ++cc) G[e++] = sW * fma(A[rr][0], A[cc][0], fma(A[rr][1], A[cc][1], A[rr][2] * A[cc][2]));
      mw = cT * W * det;
      wdet = W * det;
    }
    if (nlmode) {  // the reaction's linearised weight at this point
      const T uq = nlmode == 2 ? Ux[i] : Ur[i];
      mw = fma((nlmode == 2 ? T(3) * betaT : betaT) * wdet, uq * uq, mw);
    }
    const T Gr0 = fma(G[0], g0, fma(G[1], g1, G[2] * g2));
    const T Gr1 = fma(G[1], g0, fma(G[3], g1, G[4] * g2));
    const T Gr2 = fma(G[2], g0, fma(G[4], g1, G[5] * g2));
    const T kq = KAPPA ? io_in<T>(a.kappa_vol[(c0 + c) * M3 + q]) : T(1);
    if (DK) {
      const T *v = Ux + c * M3;
      Acc<T> b0, b1, b2;
      b0.init(tb.dcol[q0 * M], v[q1 * M + q2 * M2]);
      b1.init(tb.dcol[q1 * M], v[q0 + q2 * M2]);
      b2.init(tb.dcol[q2 * M], v[q0 + q1 * M]);
#pragma unroll
      for (int k = 1; k < M; ++k) {
        b0.add(tb.dcol[q0 * M + k], v[k + q1 * M + q2 * M2]);
        b1.add(tb.dcol[q1 * M + k], v[q0 + k * M + q2 * M2]);
        b2.add(tb.dcol[q2 * M + k], v[q0 + q1 * M + k * M2]);
      }
      const T h0 = b0.get(), h1 = b1.get(), h2 = b2.get();
      put_dk<T>(dk_vol + (c0 + c) * M3 + q, fma(Gr0, h0, fma(Gr1, h1, Gr2 * h2)), dk_acc);
    }
    F0[i] = kq * Gr0;
    F1[i] = kq * Gr1;
    F2[i] = kq * Gr2;
    MW[i] = mw;
  }
  __syncthreads();
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, q = i - c * M3;
    const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
    Acc<T> acc;
    acc.init(MW[i], Ur[i]);
    const T *f0 = F0 + c * M3, *f1 = F1 + c * M3, *f2 = F2 + c * M3;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      acc.add(tb.dcol[k * M + q0], f0[k + q1 * M + q2 * M2]);
      acc.add(tb.dcol[k * M + q1], f1[q0 + k * M + q2 * M2]);
      acc.add(tb.dcol[k * M + q2], f2[q0 + q1 * M + k * M2]);
    }
    rvol[(c0 + c) * M3 + q] = acc.get();
  }
}

template <int M, typename T>
constexpr size_t face_adj_smem(int fpb) {
  return align16<T>(sizeof(Tab<1, M, T>)) + align16<T>(fpb * sizeof(FaceId)) +
         size_t(fpb) * (13 * M * M + 72) * sizeof(T);
}

// Reference derivatives of a face trace u (M x M, qs fastest) at (qs, qt) along t1, t2.
template <int M, typename T>
__device__ __forceinline__ void tangential(const T *u, const T *dcol, int qs, int qt, T &d1, T &d2) {
  Acc<T> e1, e2;
  e1.init(dcol[qs * M], u[qt * M]);
  e2.init(dcol[qt * M], u[qs]);
#pragma unroll
  for (int k = 1; k < M; ++k) {
    e1.add(dcol[qs * M + k], u[k + qt * M]);
    e2.add(dcol[qt * M + k], u[qs + k * M]);
  }
  d1 = e1.get();
  d2 = e2.get();
}

template <int M, int GEO, bool KAPPA, bool DK, typename T>
__global__ void __launch_bounds__(256) k_face_adj(const ScalarArgs<T> a, const double theta,
                                                  const T *__restrict__ tr_r, const T *__restrict__ tr_x,
                                                  T *__restrict__ fres, io_t<T> *__restrict__ dk_face, int fpb,
                                                  bool dk_acc) {
  constexpr int M2 = M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<Tab<1, M, T> *>(smem_raw);
  // the block's faces, decoded once (64-bit divisions) and read by every point
  FaceId *sF = reinterpret_cast<FaceId *>(smem_raw + align16<T>(sizeof(Tab<1, M, T>)));
  T *SU = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(sF) + align16<T>(fpb * sizeof(FaceId)));
  T *SR = SU + fpb * 8 * M2;  // [face][5][M2]
  T *CF = SR + fpb * 5 * M2;  // [face][2 sides][36]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t f0 = (int64_t)blockIdx.x * fpb;
  const int nf = (int)min((int64_t)fpb, a.nface - f0);
  for (int i = tid; i < M * M; i += nt) tb.dcol[i] = a.tab->dcol[i];
  for (int i = tid; i < M; i += nt) { tb.w[i] = a.tab->w[i]; tb.s[i] = a.tab->s[i]; }
  for (int i = tid; i < nf; i += nt) sF[i] = decode_face(a, f0 + i);
  __syncthreads();  // faces decoded
  // stage traces: slots 0-3 r (u-, dn-, u+, dn+), 4-7 x; a boundary face uses slots of "-"
  for (int i = tid; i < nf * 8 * M2; i += nt) {
    const int lfc = i / (8 * M2), rr = i - lfc * (8 * M2);
    const int slot = rr / M2, qf = rr - slot * M2;
    const FaceId &F = sF[lfc];
    const int ax = F.axis;
    const T *tr = slot < 4 ? tr_r : tr_x;
    const int sl = slot & 3;
    T v = T(0);
    if (slot >= 4 && !DK) {
      v = T(0);
    } else if (sl < 2) {
      v = F.cm >= 0 ? tr[tr_idx<M>(F.cm, 2 * ax + 1, sl, qf)] : tr[tr_idx<M>(F.cp, 2 * ax, sl, qf)];
    } else if (F.cm >= 0 && F.cp >= 0) {
      v = tr[tr_idx<M>(F.cp, 2 * ax, sl - 2, qf)];
    }
    SU[i] = v;
  }
  if (GEO == GEO_RECOMPUTE) {
    for (int i = tid; i < nf * 2; i += nt) {
      const int lfc = i >> 1, side = i & 1;
      const FaceId &F = sF[lfc];
      int64_t cell = side == 0 ? (F.cm >= 0 ? F.cm : F.cp) : F.cp;
      if (side == 1 && (F.cm < 0 || F.cp < 0)) cell = -1;
      if (cell >= 0) {
        double V[8][3], C[3][4][3];
        dgg::cell_corners(a.verts, a.nx, a.ny, cell, V);
        dgg::jacobian_coeffs(V, C);
        for (int k = 0; k < 36; ++k) CF[i * 36 + k] = io_in<T>((&C[0][0][0])[k]);
      }
    }
  }
  __syncthreads();
  const T sc = a.sc, ss = a.ss, half = T(0.5), thetaT = io_in<T>(theta);
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const int64_t f = f0 + lfc;
    const FaceId &F = sF[lfc];
    const int ax = F.axis, t1 = F.t1, t2 = F.t2;
    const int qs = qf % M, qt = qf / M;
    const T W = tb.w[qs] * tb.w[qt];
    const bool inner = F.cm >= 0 && F.cp >= 0;
    const int side1 = F.cm >= 0 ? 1 : 0;  // xi_a of the first side (T-, or the boundary cell)
    // geometry of both sides: b (reference components) and pw
    // (arrays below are indexed with compile-time indices only, the run-time axes go
    // through selects, so that they stay in registers)
    T bm[3] = {T(0), T(0), T(0)}, bp[3] = {T(0), T(0), T(0)}, pw;
    if (GEO == GEO_AFFINE) {
      const T bW = W * a.face_b[ax];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        bm[k] = k == ax ? (inner ? bW : (side1 ? bW : -bW)) : T(0);
        bp[k] = k == ax ? bW : T(0);
      }
      pw = W * a.face_pw[ax];
    } else {
      T xi[3], J[3][3], A[3][3], n[3];
      const T xin = side1 ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) xi[k] = k == ax ? xin : (k == t1 ? tb.s[qs] : tb.s[qt]);
      dgg::jacobian_from_coeffs(CF + lfc * 72, xi[0], xi[1], xi[2], J);
      dgg::area_vector(J, ax, inner ? 1 : (side1 ? 1 : -1), n);
      T det = dgg::adjugate(J, A);
#pragma unroll
      for (int k = 0; k < 3; ++k) bm[k] = W * fma(A[k][0], n[0], fma(A[k][1], n[1], A[k][2] * n[2])) / det;
      pw = io_in<T>(a.gamma_face[f]) * W * sqrt(fma(n[0], n[0], fma(n[1], n[1], n[2] * n[2])));
      if (inner) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k == ax) xi[k] = T(0);
        dgg::jacobian_from_coeffs(CF + lfc * 72 + 36, xi[0], xi[1], xi[2], J);
        det = dgg::adjugate(J, A);
#pragma unroll
        for (int k = 0; k < 3; ++k) bp[k] = W * fma(A[k][0], n[0], fma(A[k][1], n[1], A[k][2] * n[2])) / det;
      }
    }
    const T bmn = dg_pick3(bm[0], bm[1], bm[2], ax), bm1 = dg_pick3(bm[0], bm[1], bm[2], t1);
    const T bm2 = dg_pick3(bm[0], bm[1], bm[2], t2);
    const T bpn = dg_pick3(bp[0], bp[1], bp[2], ax), bp1 = dg_pick3(bp[0], bp[1], bp[2], t1);
    const T bp2 = dg_pick3(bp[0], bp[1], bp[2], t2);
    const T *S = SU + lfc * 8 * M2;
    // b . grad_ref of r and x on each side (b given by its normal and tangential components)
    auto bgrad = [&](const T *u, const T &bn, const T &b1, const T &b2) -> T {
      T g = bn * u[M2 + qf];
      if (GEO != GEO_AFFINE) {
        T d1, d2;
        tangential<M, T>(u, tb.dcol, qs, qt, d1, d2);
        g = fma(b1, d1, fma(b2, d2, g));
      }
      return g;
    };
    const T grm = bgrad(S, bmn, bm1, bm2);
    const T gxm = DK ? bgrad(S + 4 * M2, bmn, bm1, bm2) : T(0);
    T *R = SR + lfc * 5 * M2;
    if (inner) {
      const T grp = bgrad(S + 2 * M2, bpn, bp1, bp2);
      const T gxp = DK ? bgrad(S + 6 * M2, bpn, bp1, bp2) : T(0);
      T km = T(1), kp = T(1);
      if (KAPPA) {
        km = io_in<T>(a.kappa_face[(F.cm * 6 + 2 * ax + 1) * M2 + qf]);
        kp = io_in<T>(a.kappa_face[(F.cp * 6 + 2 * ax) * M2 + qf]);
      }
      const T Jr = S[qf] - S[2 * M2 + qf];
      const T flux = half * fma(km, grm, kp * grp);
      const T Rv = fma(sc, flux, pw * Jr);
      const T sJ = ss * half * Jr;
      const T sm = KAPPA ? sJ * km : sJ, sp = KAPPA ? sJ * kp : sJ;
      fres[tr_idx<M>(F.cm, 2 * ax + 1, 1, qf)] = sm * bmn;
      fres[tr_idx<M>(F.cp, 2 * ax, 1, qf)] = sp * bpn;
      if (GEO == GEO_AFFINE) {
        fres[tr_idx<M>(F.cm, 2 * ax + 1, 0, qf)] = Rv;
        fres[tr_idx<M>(F.cp, 2 * ax, 0, qf)] = -Rv;
      } else {
        R[qf] = Rv;
        R[M2 + qf] = sm * bm1;
        R[2 * M2 + qf] = sm * bm2;
        R[3 * M2 + qf] = sp * bp1;
        R[4 * M2 + qf] = sp * bp2;
      }
      if (DK) {
        const T Jx = S[4 * M2 + qf] - S[6 * M2 + qf];
        put_dk<T>(dk_face + (F.cm * 6 + 2 * ax + 1) * M2 + qf, half * fma(-gxm, Jr, thetaT * Jx * grm), dk_acc);
        put_dk<T>(dk_face + (F.cp * 6 + 2 * ax) * M2 + qf, half * fma(-gxp, Jr, thetaT * Jx * grp), dk_acc);
      }
    } else {
      const int64_t cb = side1 ? F.cm : F.cp;
      const int lf = 2 * ax + side1;
      T Rv = T(0), s1 = T(0), s2 = T(0), sn = T(0), dk = T(0);
      if ((a.dmask >> lf) & 1u) {
        const T kb = KAPPA ? io_in<T>(a.kappa_face[(cb * 6 + lf) * M2 + qf]) : T(1);
        const T u = S[qf];
        Rv = fma(sc * kb, grm, pw * u);
        const T su = ss * kb * u;
        s1 = su * bm1;
        s2 = su * bm2;
        sn = su * bmn;
        if (DK) dk = fma(-gxm, u, thetaT * S[4 * M2 + qf] * grm);
      }
      fres[tr_idx<M>(cb, lf, 1, qf)] = sn;
      if (GEO == GEO_AFFINE) {
        fres[tr_idx<M>(cb, lf, 0, qf)] = Rv;
      } else {
        R[qf] = Rv;
        R[M2 + qf] = s1;
        R[2 * M2 + qf] = s2;
      }
      if (DK) put_dk<T>(dk_face + (cb * 6 + lf) * M2 + qf, dk, dk_acc);
    }
  }
  if (GEO == GEO_AFFINE) return;
  __syncthreads();
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const FaceId &F = sF[lfc];
    const int ax = F.axis;
    const int qs = qf % M, qt = qf / M;
    const T *R = SR + lfc * 5 * M2;
    Acc<T> vm;
    vm.set(R[qf]);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      vm.add(tb.dcol[k * M + qs], R[M2 + k + qt * M]);
      vm.add(tb.dcol[k * M + qt], R[2 * M2 + qs + k * M]);
    }
    if (F.cm >= 0 && F.cp >= 0) {
      Acc<T> vp;
      vp.set(-R[qf]);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        vp.add(tb.dcol[k * M + qs], R[3 * M2 + k + qt * M]);
        vp.add(tb.dcol[k * M + qt], R[4 * M2 + qs + k * M]);
      }
      fres[tr_idx<M>(F.cm, 2 * ax + 1, 0, qf)] = vm.get();
      fres[tr_idx<M>(F.cp, 2 * ax, 0, qf)] = vp.get();
    } else {
      const int side = F.cm >= 0 ? 1 : 0;
      fres[tr_idx<M>(side ? F.cm : F.cp, 2 * ax + side, 0, qf)] = vm.get();
    }
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

template <int P, int GEO, bool KAPPA, bool DK, typename T>
cudaError_t run(const ScalarArgs<T> &a, double theta, const io_t<T> *r, const io_t<T> *x, io_t<T> *y,
                io_t<T> *dk_vol, io_t<T> *dk_face, T *rvol, T *tr_r, T *tr_x, T *fres, int cpb, int fpb,
                cudaStream_t s, const cudaEvent_t *ev, int nlmode, double beta, bool dk_acc) {
  constexpr int M = P, M2 = M * M, M3 = M * M * M;
  cudaError_t e;
  {
    const size_t sm = cell_adj_smem<P, M, T>(cpb);
    auto k = k_cell_adj<P, GEO, KAPPA, DK, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    k<<<(unsigned)((a.ncell + cpb - 1) / cpb), threads_for(cpb * M3), sm, s>>>(a, r, x, rvol, tr_r, tr_x, dk_vol, cpb,
                                                                              nlmode, beta, dk_acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const size_t sm = face_adj_smem<M, T>(fpb);
    auto k = k_face_adj<M, GEO, KAPPA, DK, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    k<<<(unsigned)((a.nface + fpb - 1) / fpb), threads_for(fpb * M2), sm, s>>>(a, theta, tr_r, tr_x, fres, dk_face, fpb, dk_acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const size_t sm = back_smem_bytes<P, M, T>(cpb);
    auto k = k_back<P, M, T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], s);
    k<<<dim3((unsigned)((a.ncell + cpb - 1) / cpb), 1), threads_for(cpb * M3), sm, s>>>(a, rvol, fres, y, cpb, 0, 0, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], s);
  }
  return cudaSuccess;
}

template <int P, typename T>
cudaError_t run_p(int geo, bool kappa, bool dk, const ScalarArgs<T> &a, double theta, const io_t<T> *r,
                  const io_t<T> *x, io_t<T> *y, io_t<T> *dkv, io_t<T> *dkf, T *rvol, T *trr, T *trx, T *fres, int cpb,
                  int fpb, cudaStream_t s, const cudaEvent_t *ev, int nlmode, double beta, bool dk_acc) {
#define DGA_RUN(G, K, D) \
  return run<P, G, K, D, T>(a, theta, r, x, y, dkv, dkf, rvol, trr, trx, fres, cpb, fpb, s, ev, nlmode, beta, dk_acc)
  if (geo == GEO_AFFINE) {
    if (kappa) { if (dk) DGA_RUN(GEO_AFFINE, true, true); DGA_RUN(GEO_AFFINE, true, false); }
    if (dk) DGA_RUN(GEO_AFFINE, false, true);
    DGA_RUN(GEO_AFFINE, false, false);
  }
  if (kappa) { if (dk) DGA_RUN(GEO_RECOMPUTE, true, true); DGA_RUN(GEO_RECOMPUTE, true, false); }
  if (dk) DGA_RUN(GEO_RECOMPUTE, false, true);
  DGA_RUN(GEO_RECOMPUTE, false, false);
#undef DGA_RUN
}

}  // namespace dga

template <typename T>
cudaError_t launch_scalar_adjoint(int p, int geo, bool kappa, const ScalarArgs<T> &a, double theta, const io_t<T> *r,
                                  const io_t<T> *x, io_t<T> *y, io_t<T> *dk_vol, io_t<T> *dk_face, T *rvol, T *tr_r,
                                  T *tr_x, T *fres, int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev,
                                  int nlmode, double beta, bool dk_acc) {
  const bool dk = x != nullptr && dk_vol != nullptr && dk_face != nullptr;
  if ((nlmode == 2 && !x) || (nlmode && dk)) return cudaErrorInvalidValue;
  switch (p) {
#define DGA_P(PP)                                                                                                \
  case PP:                                                                                                       \
    return dga::run_p<PP, T>(geo, kappa, dk, a, theta, r, x, y, dk_vol, dk_face, rvol, tr_r, tr_x, fres, cpb, fpb, s, \
                             ev, nlmode, beta, dk_acc);
    DGA_P(2) DGA_P(3) DGA_P(4) DGA_P(5) DGA_P(6)
#undef DGA_P
    default: return cudaErrorInvalidValue;
  }
}
