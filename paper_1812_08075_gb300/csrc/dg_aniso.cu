// Scalar SIPG apply with anisotropic degrees and quadrature (Sec. 2.1: a degree k_a and a
// Gauss rule of m_a points per direction; Sec. 4 raises m on purpose): the three-kernel
// structure of the isotropic apply with run-time extents. Direction a has p_a = k_a + 1
// GLL basis points and m_a >= p_a Gauss points.
//   k_an_cell: interpolation to the Gauss points one direction at a time (Algorithm 1:
//     p2 p1 p0 -> p2 p1 m0 -> p2 m1 m0 -> m2 m1 m0 values), the traces of the six faces
//     (face normal to a: m_t1 x m_t2 points), the gradient, the pointwise flux kappa G grad
//     (affine: diagonal metric; trilinear: G = W detJ J^-1 J^-T recomputed from the vertex
//     coordinates at every point), the mass term and the transposed derivative.
//   k_an_face: per face, the jump, average flux and penalty from both sides' traces
//     (Eq. diffreac_weak); on curved faces the tangential derivatives of the traces enter
//     the flux and the symmetry term, whose tangential parts are lifted by a transposed
//     tangential derivative; written as each side's (value, normal-derivative) residuals.
//   k_an_back: lifting of the face residuals and the transposed interpolation.
// Per cell the traces and face residuals are [6 faces][2][m_t1 m_t2] with per-face offsets;
// kappa is kappa_vol [ncell][m0 m1 m2] and kappa_face [ncell][sum over faces of m_t1 m_t2].
#include <string.h>

#include <vector>

#include "dg_geo_device.cuh"
#include "dg_scalar_kernels.cuh"

namespace dgn {

using dgk::decode_face;
using dgk::FaceId;

template <typename T>
struct AnTab {
  int p[3], m[3];
  int toff[7];  // offset of face lf's (value, derivative) pair in a cell's trace block; toff[6] = size
  int foff[7];  // offset of face lf's points in a cell's kappa_face block; foff[6] = size
  T interp[3][DG_MAXM * DG_MAXP];  // [a][q * p_a + j]
  T dcol[3][DG_MAXM * DG_MAXM];    // [a][q * m_a + r]
  T e0[3][DG_MAXM], e1[3][DG_MAXM], d0[3][DG_MAXM], d1[3][DG_MAXM], w[3][DG_MAXM], s[3][DG_MAXM];
};

__host__ __device__ inline void tangential(int a, int &t1, int &t2) {
  t1 = a == 0 ? 1 : 0;
  t2 = a == 2 ? 1 : 2;
}

// Index of the point with coordinate r along axis a and (s, t) along its tangential axes.
__device__ __forceinline__ int pidx(const int *m, int a, int r, int s, int t) {
  int q[3];
  int t1, t2;
  tangential(a, t1, t2);
  q[a] = r;
  q[t1] = s;
  q[t2] = t;
  return q[0] + m[0] * (q[1] + m[1] * q[2]);
}

template <typename T>
__device__ void stage_tab(AnTab<T> &s, const AnTab<T> *g) {
  const int *src = reinterpret_cast<const int *>(g);
  int *dst = reinterpret_cast<int *>(&s);
  for (int i = threadIdx.x; i < (int)(sizeof(AnTab<T>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
}

// Per cell: six buffers of N = m0 m1 m2 values (the interpolation stages fit in N because
// m_a >= p_a) and the 36 coefficients of the trilinear Jacobian.
template <typename T>
inline size_t an_cell_smem(int cpb, int N) {
  return (size_t)cpb * (6 * (size_t)N + 36) * sizeof(T);
}

template <typename T, int GEO, bool KAPPA>
__global__ void __launch_bounds__(256) k_an_cell(const ScalarArgs<T> a, const AnTab<T> *__restrict__ gtab,
                                                 const T *__restrict__ x, T *__restrict__ rvol,
                                                 T *__restrict__ traces, int cpb, int64_t sdof, int64_t srv,
                                                 int64_t str) {
  __shared__ AnTab<T> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_tab(tb, gtab);
  __syncthreads();
  const int *m = tb.m, *p = tb.p;
  const int N = m[0] * m[1] * m[2], P = p[0] * p[1] * p[2], TS = tb.toff[6];
  T *A = reinterpret_cast<T *>(smem_raw), *B = A + cpb * N, *U = B + cpb * N;
  T *F0 = U + cpb * N, *F1 = F0 + cpb * N, *F2 = F1 + cpb * N, *CC = F2 + cpb * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  x += blockIdx.y * sdof;
  rvol += blockIdx.y * srv;
  traces += blockIdx.y * str;
  for (int i = tid; i < nc * P; i += nt) {
    const int c = i / P;
    A[c * N + (i - c * P)] = x[c0 * P + i];
  }
  if (GEO == GEO_RECOMPUTE) {
    for (int c = tid; c < nc; c += nt) {
      double V[8][3], C[3][4][3];
      dgg::cell_corners(a.verts, a.nx, a.ny, c0 + c, V);
      dgg::jacobian_coeffs(V, C);
      for (int k = 0; k < 36; ++k) CC[c * 36 + k] = (T)((&C[0][0][0])[k]);
    }
  }
  __syncthreads();
  // interpolation: x-sweep A [j0 + p0 (j1 + p1 j2)] -> B [q0 + m0 (j1 + p1 j2)]
  const int S1 = m[0] * p[1] * p[2], S2 = m[0] * m[1] * p[2];
  for (int i = tid; i < nc * S1; i += nt) {
    const int c = i / S1, r = i - c * S1, q0 = r % m[0], j12 = r / m[0];
    const T *src = A + c * N + j12 * p[0];
    T s = T(0);
    for (int j = 0; j < p[0]; ++j) s = fma(tb.interp[0][q0 * p[0] + j], src[j], s);
    B[c * N + r] = s;
  }
  __syncthreads();
  // y-sweep B -> A [q0 + m0 (q1 + m1 j2)]
  for (int i = tid; i < nc * S2; i += nt) {
    const int c = i / S2, r = i - c * S2, q0 = r % m[0], q1 = (r / m[0]) % m[1], j2 = r / (m[0] * m[1]);
    const T *src = B + c * N + q0 + m[0] * p[1] * j2;
    T s = T(0);
    for (int j = 0; j < p[1]; ++j) s = fma(tb.interp[1][q1 * p[1] + j], src[j * m[0]], s);
    A[c * N + r] = s;
  }
  __syncthreads();
  // z-sweep A -> U [q0 + m0 (q1 + m1 q2)]
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, r = i - c * N, q01 = r % (m[0] * m[1]), q2 = r / (m[0] * m[1]);
    const T *src = A + c * N + q01;
    T s = T(0);
    for (int j = 0; j < p[2]; ++j) s = fma(tb.interp[2][q2 * p[2] + j], src[j * m[0] * m[1]], s);
    U[i] = s;
  }
  __syncthreads();
  // traces of the six faces: (value, reference normal derivative) at the face points
  for (int i = tid; i < nc * TS; i += nt) {
    const int c = i / TS, r = i - c * TS;
    int lf = 0;
    while (r >= tb.toff[lf + 1]) ++lf;
    const int ax = lf >> 1, side = lf & 1;
    int t1, t2;
    tangential(ax, t1, t2);
    const int F = m[t1] * m[t2], o = r - tb.toff[lf], qty = o / F, qf = o - qty * F;
    const int qs = qf % m[t1], qt = qf / m[t1];
    const T *row = side ? (qty ? tb.d1[ax] : tb.e1[ax]) : (qty ? tb.d0[ax] : tb.e0[ax]);
    T s = T(0);
    for (int k = 0; k < m[ax]; ++k) s = fma(row[k], U[c * N + pidx(m, ax, k, qs, qt)], s);
    traces[(c0 + c) * TS + r] = s;
  }
  // gradient, pointwise flux kappa G grad and mass term
  const T cT = (T)a.c;
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, q = i - c * N;
    const int q0 = q % m[0], q1 = (q / m[0]) % m[1], q2 = q / (m[0] * m[1]);
    const T *u = U + c * N;
    T g0 = T(0), g1 = T(0), g2 = T(0);
    for (int k = 0; k < m[0]; ++k) g0 = fma(tb.dcol[0][q0 * m[0] + k], u[k + m[0] * (q1 + m[1] * q2)], g0);
    for (int k = 0; k < m[1]; ++k) g1 = fma(tb.dcol[1][q1 * m[1] + k], u[q0 + m[0] * (k + m[1] * q2)], g1);
    for (int k = 0; k < m[2]; ++k) g2 = fma(tb.dcol[2][q2 * m[2] + k], u[q0 + m[0] * (q1 + m[1] * k)], g2);
    const T W = tb.w[0][q0] * tb.w[1][q1] * tb.w[2][q2];
    const T kq = KAPPA ? (T)a.kappa_vol[(c0 + c) * N + q] : T(1);
    if (GEO == GEO_AFFINE) {
      F0[i] = kq * W * a.vol_g[0] * g0;
      F1[i] = kq * W * a.vol_g[1] * g1;
      F2[i] = kq * W * a.vol_g[2] * g2;
      B[i] = W * a.vol_m * u[q];
    } else {
      T J[3][3], Ad[3][3];
      dgg::jacobian_from_coeffs(CC + c * 36, tb.s[0][q0], tb.s[1][q1], tb.s[2][q2], J);
      const T det = dgg::adjugate(J, Ad);
      const T sW = kq * W / det;
      T G[3][3];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) G[rr][cc] = sW * fma(Ad[rr][0], Ad[cc][0], fma(Ad[rr][1], Ad[cc][1], Ad[rr][2] * Ad[cc][2]));
      F0[i] = fma(G[0][0], g0, fma(G[0][1], g1, G[0][2] * g2));
      F1[i] = fma(G[1][0], g0, fma(G[1][1], g1, G[1][2] * g2));
      F2[i] = fma(G[2][0], g0, fma(G[2][1], g1, G[2][2] * g2));
      B[i] = cT * W * det * u[q];
    }
  }
  __syncthreads();
  // transposed derivative -> Gauss-point residual
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, q = i - c * N;
    const int q0 = q % m[0], q1 = (q / m[0]) % m[1], q2 = q / (m[0] * m[1]);
    const T *f0 = F0 + c * N, *f1 = F1 + c * N, *f2 = F2 + c * N;
    T s = B[i];
    for (int k = 0; k < m[0]; ++k) s = fma(tb.dcol[0][k * m[0] + q0], f0[k + m[0] * (q1 + m[1] * q2)], s);
    for (int k = 0; k < m[1]; ++k) s = fma(tb.dcol[1][k * m[1] + q1], f1[q0 + m[0] * (k + m[1] * q2)], s);
    for (int k = 0; k < m[2]; ++k) s = fma(tb.dcol[2][k * m[2] + q2], f2[q0 + m[0] * (q1 + m[1] * k)], s);
    rvol[(c0 + c) * N + q] = s;
  }
}

constexpr int MF = DG_MAXM * DG_MAXM;  // face points, at most

// Per face: its decoded id, both sides' (value, normal derivative) traces [4][MF], five
// residual components [5][MF] (curved faces) and both cells' Jacobian coefficients.
template <typename T>
inline size_t an_face_smem(int fpb) {
  return dgk::align16<T>((size_t)fpb * sizeof(FaceId)) + (size_t)fpb * (9 * MF + 72) * sizeof(T);
}

template <typename T, int GEO, bool KAPPA>
__global__ void __launch_bounds__(256) k_an_face(const ScalarArgs<T> a, const AnTab<T> *__restrict__ gtab,
                                                 const T *__restrict__ traces, T *__restrict__ fres, int fpb,
                                                 int64_t str) {
  __shared__ AnTab<T> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FaceId *sF = reinterpret_cast<FaceId *>(smem_raw);
  T *SU = reinterpret_cast<T *>(smem_raw + dgk::align16<T>((size_t)fpb * sizeof(FaceId)));
  T *SR = SU + fpb * 4 * MF;
  T *CF = SR + fpb * 5 * MF;
  stage_tab(tb, gtab);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t f0 = (int64_t)blockIdx.x * fpb;
  const int nf = (int)min((int64_t)fpb, a.nface - f0);
  for (int i = tid; i < nf; i += nt) sF[i] = decode_face(a, f0 + i);
  __syncthreads();
  const int *m = tb.m;
  const int TS = tb.toff[6], NF = tb.foff[6];
  traces += blockIdx.y * str;
  fres += blockIdx.y * str;
  // stage traces: slots 0-1 the "-" side (or the boundary cell), 2-3 the "+" side
  for (int i = tid; i < nf * 4 * MF; i += nt) {
    const int lfc = i / (4 * MF), rr = i - lfc * 4 * MF, slot = rr / MF, qf = rr - slot * MF;
    const FaceId &Fc = sF[lfc];
    const int ax = Fc.axis, F = m[Fc.t1] * m[Fc.t2];
    if (qf >= F) continue;
    T v = T(0);
    if (slot < 2)
      v = Fc.cm >= 0 ? traces[Fc.cm * TS + tb.toff[2 * ax + 1] + slot * F + qf]
                     : traces[Fc.cp * TS + tb.toff[2 * ax] + slot * F + qf];
    else if (Fc.cm >= 0 && Fc.cp >= 0)
      v = traces[Fc.cp * TS + tb.toff[2 * ax] + (slot - 2) * F + qf];
    SU[i] = v;
  }
  if (GEO == GEO_RECOMPUTE) {
    for (int i = tid; i < nf * 2; i += nt) {
      const int lfc = i >> 1, side = i & 1;
      const FaceId &Fc = sF[lfc];
      int64_t cell = side == 0 ? (Fc.cm >= 0 ? Fc.cm : Fc.cp) : Fc.cp;
      if (side == 1 && (Fc.cm < 0 || Fc.cp < 0)) cell = -1;
      if (cell >= 0) {
        double V[8][3], C[3][4][3];
        dgg::cell_corners(a.verts, a.nx, a.ny, cell, V);
        dgg::jacobian_coeffs(V, C);
        for (int k = 0; k < 36; ++k) CF[i * 36 + k] = (T)((&C[0][0][0])[k]);
      }
    }
  }
  __syncthreads();
  const T sc = a.sc, ss = a.ss, half = T(0.5);
  for (int i = tid; i < nf * MF; i += nt) {
    const int lfc = i / MF, qf = i - lfc * MF;
    const FaceId &Fc = sF[lfc];
    const int ax = Fc.axis, t1 = Fc.t1, t2 = Fc.t2, mt1 = m[t1], mt2 = m[t2], F = mt1 * mt2;
    if (qf >= F) continue;
    const int64_t f = f0 + lfc;
    const int qs = qf % mt1, qt = qf / mt1;
    const T W = tb.w[t1][qs] * tb.w[t2][qt];
    const bool inner = Fc.cm >= 0 && Fc.cp >= 0;
    const int side1 = Fc.cm >= 0 ? 1 : 0;  // xi_a of the first side (T-, or the boundary cell)
    T bm[3] = {T(0), T(0), T(0)}, bp[3] = {T(0), T(0), T(0)}, pw;
    if (GEO == GEO_AFFINE) {
      const T bW = W * a.face_b[ax];
      bm[ax] = inner ? bW : (side1 ? bW : -bW);
      bp[ax] = bW;
      pw = W * a.face_pw[ax];
    } else {
      T xi[3], J[3][3], Ad[3][3], n[3];
      xi[t1] = tb.s[t1][qs];
      xi[t2] = tb.s[t2][qt];
      xi[ax] = side1 ? T(1) : T(0);
      dgg::jacobian_from_coeffs(CF + lfc * 72, xi[0], xi[1], xi[2], J);
      dgg::area_vector(J, ax, inner ? 1 : (side1 ? 1 : -1), n);
      T det = dgg::adjugate(J, Ad);
#pragma unroll
      for (int k = 0; k < 3; ++k) bm[k] = W * fma(Ad[k][0], n[0], fma(Ad[k][1], n[1], Ad[k][2] * n[2])) / det;
      pw = (T)a.gamma_face[f] * W * sqrt(fma(n[0], n[0], fma(n[1], n[1], n[2] * n[2])));
      if (inner) {
        xi[ax] = T(0);
        dgg::jacobian_from_coeffs(CF + lfc * 72 + 36, xi[0], xi[1], xi[2], J);
        det = dgg::adjugate(J, Ad);
#pragma unroll
        for (int k = 0; k < 3; ++k) bp[k] = W * fma(Ad[k][0], n[0], fma(Ad[k][1], n[1], Ad[k][2] * n[2])) / det;
      }
    }
    const T *S = SU + lfc * 4 * MF;
    // b . grad_ref u on one side (u: that side's trace values, normal derivative at +MF)
    auto bgrad = [&](const T *u, const T *b) -> T {
      T g = b[ax] * u[MF + qf];
      if (GEO != GEO_AFFINE) {
        T d1 = T(0), d2 = T(0);
        for (int k = 0; k < mt1; ++k) d1 = fma(tb.dcol[t1][qs * mt1 + k], u[k + mt1 * qt], d1);
        for (int k = 0; k < mt2; ++k) d2 = fma(tb.dcol[t2][qt * mt2 + k], u[qs + mt1 * k], d2);
        g = fma(b[t1], d1, fma(b[t2], d2, g));
      }
      return g;
    };
    const T gm = bgrad(S, bm);
    T *R = SR + lfc * 5 * MF;
    if (inner) {
      const T gp = bgrad(S + 2 * MF, bp);
      T km = T(1), kp = T(1);
      if (KAPPA) {
        km = (T)a.kappa_face[Fc.cm * NF + tb.foff[2 * ax + 1] + qf];
        kp = (T)a.kappa_face[Fc.cp * NF + tb.foff[2 * ax] + qf];
      }
      const T Jr = S[qf] - S[2 * MF + qf];
      const T flux = half * fma(km, gm, kp * gp);
      const T Rv = fma(sc, flux, pw * Jr);
      const T sJ = ss * half * Jr;
      const T sm = KAPPA ? sJ * km : sJ, sp = KAPPA ? sJ * kp : sJ;
      const int64_t om = Fc.cm * TS + tb.toff[2 * ax + 1], op = Fc.cp * TS + tb.toff[2 * ax];
      fres[om + F + qf] = sm * bm[ax];
      fres[op + F + qf] = sp * bp[ax];
      if (GEO == GEO_AFFINE) {
        fres[om + qf] = Rv;
        fres[op + qf] = -Rv;
      } else {
        R[qf] = Rv;
        R[MF + qf] = sm * bm[t1];
        R[2 * MF + qf] = sm * bm[t2];
        R[3 * MF + qf] = sp * bp[t1];
        R[4 * MF + qf] = sp * bp[t2];
      }
    } else {
      const int64_t cb = side1 ? Fc.cm : Fc.cp;
      const int lf = 2 * ax + side1;
      T Rv = T(0), s1 = T(0), s2 = T(0), sn = T(0);
      if ((a.dmask >> lf) & 1u) {
        const T kb = KAPPA ? (T)a.kappa_face[cb * NF + tb.foff[lf] + qf] : T(1);
        const T u = S[qf];
        Rv = fma(sc * kb, gm, pw * u);
        const T su = ss * kb * u;
        s1 = su * bm[t1];
        s2 = su * bm[t2];
        sn = su * bm[ax];
      }
      const int64_t ob = cb * TS + tb.toff[lf];
      fres[ob + F + qf] = sn;
      if (GEO == GEO_AFFINE) {
        fres[ob + qf] = Rv;
      } else {
        R[qf] = Rv;
        R[MF + qf] = s1;
        R[2 * MF + qf] = s2;
      }
    }
  }
  if (GEO == GEO_AFFINE) return;
  __syncthreads();
  // curved faces: the symmetry term's tangential parts through the transposed tangential
  // derivative, added to each side's value residual
  for (int i = tid; i < nf * MF; i += nt) {
    const int lfc = i / MF, qf = i - lfc * MF;
    const FaceId &Fc = sF[lfc];
    const int ax = Fc.axis, t1 = Fc.t1, t2 = Fc.t2, mt1 = m[t1], mt2 = m[t2], F = mt1 * mt2;
    if (qf >= F) continue;
    const int qs = qf % mt1, qt = qf / mt1;
    const T *R = SR + lfc * 5 * MF;
    T vm = R[qf];
    for (int k = 0; k < mt1; ++k) vm = fma(tb.dcol[t1][k * mt1 + qs], R[MF + k + mt1 * qt], vm);
    for (int k = 0; k < mt2; ++k) vm = fma(tb.dcol[t2][k * mt2 + qt], R[2 * MF + qs + mt1 * k], vm);
    if (Fc.cm >= 0 && Fc.cp >= 0) {
      T vp = -R[qf];
      for (int k = 0; k < mt1; ++k) vp = fma(tb.dcol[t1][k * mt1 + qs], R[3 * MF + k + mt1 * qt], vp);
      for (int k = 0; k < mt2; ++k) vp = fma(tb.dcol[t2][k * mt2 + qt], R[4 * MF + qs + mt1 * k], vp);
      fres[Fc.cm * TS + tb.toff[2 * ax + 1] + qf] = vm;
      fres[Fc.cp * TS + tb.toff[2 * ax] + qf] = vp;
    } else {
      const int side = Fc.cm >= 0 ? 1 : 0;
      fres[(side ? Fc.cm : Fc.cp) * TS + tb.toff[2 * ax + side] + qf] = vm;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_an_back(const ScalarArgs<T> a, const AnTab<T> *__restrict__ gtab,
                                                 const T *__restrict__ rvol, const T *__restrict__ fres,
                                                 T *__restrict__ y, int cpb, int64_t sdof, int64_t srv,
                                                 int64_t str) {
  __shared__ AnTab<T> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_tab(tb, gtab);
  __syncthreads();
  const int *m = tb.m, *p = tb.p;
  const int N = m[0] * m[1] * m[2], P = p[0] * p[1] * p[2], TS = tb.toff[6];
  T *A = reinterpret_cast<T *>(smem_raw), *B = A + cpb * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  rvol += blockIdx.y * srv;
  fres += blockIdx.y * str;
  y += blockIdx.y * sdof;
  // Gauss-point residual with the lifted face residuals of the six faces
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, q = i - c * N;
    const int qq[3] = {q % m[0], (q / m[0]) % m[1], q / (m[0] * m[1])};
    const T *fr = fres + (c0 + c) * TS;
    T s = rvol[(c0 + c) * N + q];
    for (int ax = 0; ax < 3; ++ax) {
      int t1, t2;
      tangential(ax, t1, t2);
      const int F = m[t1] * m[t2], qf = qq[t1] + m[t1] * qq[t2], r = qq[ax];
      const T *lo = fr + tb.toff[2 * ax], *hi = fr + tb.toff[2 * ax + 1];
      s = fma(tb.e0[ax][r], lo[qf], s);
      s = fma(tb.d0[ax][r], lo[F + qf], s);
      s = fma(tb.e1[ax][r], hi[qf], s);
      s = fma(tb.d1[ax][r], hi[F + qf], s);
    }
    A[i] = s;
  }
  __syncthreads();
  // transposed interpolation: z (A [q0 + m0 (q1 + m1 q2)] -> B [q0 + m0 (q1 + m1 j2)]),
  // y (B -> A [q0 + m0 (j1 + p1 j2)]), x (A -> y [j0 + p0 (j1 + p1 j2)])
  const int S2 = m[0] * m[1] * p[2], S1 = m[0] * p[1] * p[2];
  for (int i = tid; i < nc * S2; i += nt) {
    const int c = i / S2, r = i - c * S2, q01 = r % (m[0] * m[1]), j2 = r / (m[0] * m[1]);
    const T *src = A + c * N + q01;
    T s = T(0);
    for (int q = 0; q < m[2]; ++q) s = fma(tb.interp[2][q * p[2] + j2], src[q * m[0] * m[1]], s);
    B[c * N + r] = s;
  }
  __syncthreads();
  for (int i = tid; i < nc * S1; i += nt) {
    const int c = i / S1, r = i - c * S1, q0 = r % m[0], j1 = (r / m[0]) % p[1], j2 = r / (m[0] * p[1]);
    const T *src = B + c * N + q0 + m[0] * m[1] * j2;
    T s = T(0);
    for (int q = 0; q < m[1]; ++q) s = fma(tb.interp[1][q * p[1] + j1], src[q * m[0]], s);
    A[c * N + r] = s;
  }
  __syncthreads();
  for (int i = tid; i < nc * P; i += nt) {
    const int c = i / P, r = i - c * P, j0 = r % p[0], j12 = r / p[0];
    const T *src = A + c * N + j12 * m[0];
    T s = T(0);
    for (int q = 0; q < m[0]; ++q) s = fma(tb.interp[0][q * p[0] + j0], src[q], s);
    y[(c0 + c) * P + r] = s;
  }
}

inline int threads_for(int work) {
  const int t = ((work + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

template <typename T, int GEO, bool KAPPA>
cudaError_t run(const ScalarArgs<T> &a, const AnTab<T> *tab, int npts, int nq, const T *x, T *y, T *rvol,
                T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str, int cpb, int fpb,
                cudaStream_t s, const cudaEvent_t *ev) {
  cudaError_t e;
  const size_t smc = an_cell_smem<T>(cpb, nq), smf = an_face_smem<T>(fpb), smb = (size_t)cpb * 2 * nq * sizeof(T);
  if ((e = set_smem(k_an_cell<T, GEO, KAPPA>, smc)) != cudaSuccess) return e;
  if ((e = set_smem(k_an_face<T, GEO, KAPPA>, smf)) != cudaSuccess) return e;
  if ((e = set_smem(k_an_back<T>, smb)) != cudaSuccess) return e;
  const dim3 gc((unsigned)((a.ncell + cpb - 1) / cpb), nrhs), gf((unsigned)((a.nface + fpb - 1) / fpb), nrhs);
  if (ev) cudaEventRecord(ev[0], s);
  k_an_cell<T, GEO, KAPPA><<<gc, threads_for(cpb * nq), smc, s>>>(a, tab, x, rvol, traces, cpb, sdof, srv, str);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  k_an_face<T, GEO, KAPPA><<<gf, threads_for(fpb * MF), smf, s>>>(a, tab, traces, fres, fpb, str);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  k_an_back<T><<<gc, threads_for(cpb * nq), smb, s>>>(a, tab, rvol, fres, y, cpb, sdof, srv, str);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  return cudaSuccess;
}

}  // namespace dgn

// Host side: tables of the three directions (each direction's own 1D tables for its k_a and
// m_a), the trace offsets and the kappa_face offsets. host_tab: aniso_tab_bytes<T>() bytes.
template <typename T>
size_t aniso_tab_bytes() {
  return sizeof(dgn::AnTab<T>);
}

template <typename T>
int aniso_tables(const HostTables ht[3], void *host_tab, int *trace_size) {
  dgn::AnTab<T> &t = *reinterpret_cast<dgn::AnTab<T> *>(host_tab);
  memset(&t, 0, sizeof(t));
  for (int a = 0; a < 3; ++a) {
    const HostTables &h = ht[a];
    if (h.m < h.p) return -1;
    t.p[a] = h.p;
    t.m[a] = h.m;
    for (int i = 0; i < h.m * h.p; ++i) t.interp[a][i] = (T)h.interp[i];
    for (int i = 0; i < h.m * h.m; ++i) t.dcol[a][i] = (T)h.dcol[i];
    for (int i = 0; i < h.m; ++i) {
      t.e0[a][i] = (T)h.e0[i]; t.e1[a][i] = (T)h.e1[i];
      t.d0[a][i] = (T)h.d0[i]; t.d1[a][i] = (T)h.d1[i];
      t.w[a][i] = (T)h.gauss_w[i]; t.s[a][i] = (T)h.gauss_s[i];
    }
  }
  int off = 0;
  for (int lf = 0; lf < 6; ++lf) {
    int t1, t2;
    dgn::tangential(lf >> 1, t1, t2);
    t.toff[lf] = off;
    t.foff[lf] = off / 2;
    off += 2 * t.m[t1] * t.m[t2];
  }
  t.toff[6] = off;
  t.foff[6] = off / 2;
  *trace_size = off;
  return 0;
}

template <typename T>
cudaError_t launch_aniso_apply(const ScalarArgs<T> &a, const void *dtab, int npts, int trace_size, const T *x, T *y,
                               T *rvol, T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str,
                               int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev, int geo, bool kappa,
                               int nq) {
  using namespace dgn;
  (void)trace_size;
  const AnTab<T> *tab = reinterpret_cast<const AnTab<T> *>(dtab);
#define DGN_RUN(G, K) return run<T, G, K>(a, tab, npts, nq, x, y, rvol, traces, fres, nrhs, sdof, srv, str, cpb, fpb, s, ev)
  if (geo == GEO_AFFINE) {
    if (kappa) DGN_RUN(GEO_AFFINE, true);
    DGN_RUN(GEO_AFFINE, false);
  }
  if (kappa) DGN_RUN(GEO_RECOMPUTE, true);
  DGN_RUN(GEO_RECOMPUTE, false);
#undef DGN_RUN
}

template size_t aniso_tab_bytes<double>();
template size_t aniso_tab_bytes<float>();
template int aniso_tables<double>(const HostTables[3], void *, int *);
template int aniso_tables<float>(const HostTables[3], void *, int *);
template cudaError_t launch_aniso_apply<double>(const ScalarArgs<double> &, const void *, int, int, const double *,
                                                double *, double *, double *, double *, int, int64_t, int64_t,
                                                int64_t, int, int, cudaStream_t, const cudaEvent_t *, int, bool, int);
template cudaError_t launch_aniso_apply<float>(const ScalarArgs<float> &, const void *, int, int, const float *,
                                               float *, float *, float *, float *, int, int64_t, int64_t, int64_t,
                                               int, int, cudaStream_t, const cudaEvent_t *, int, bool, int);

// Operation counts of the three kernels (FMA = 2; with recomputed trilinear geometry the
// per-point Jacobian, adjugate and metric are counted as 156 flops per volume point and
// about 250 per face point, two sides) and their algorithmic bytes.
void aniso_work_model(const int kax[3], const int max[3], int geo, bool kappa, int64_t ncell, int64_t nface,
                      int64_t nbface, double flops[3], double bytes[3], int es) {
  const double p[3] = {kax[0] + 1.0, kax[1] + 1.0, kax[2] + 1.0};
  const double m[3] = {(double)max[0], (double)max[1], (double)max[2]};
  const double N = m[0] * m[1] * m[2], P = p[0] * p[1] * p[2];
  const double S1 = m[0] * p[1] * p[2], S2 = m[0] * m[1] * p[2];
  const double F[3] = {m[1] * m[2], m[0] * m[2], m[0] * m[1]};  // face points normal to each axis
  const bool tri = geo != GEO_AFFINE;
  double cell = 2.0 * (S1 * p[0] + S2 * p[1] + N * p[2]);  // interpolation
  double ts = 0.0, fsum = 0.0;
  for (int a = 0; a < 3; ++a) {
    cell += 2.0 * 2.0 * F[a] * 2.0 * m[a];  // traces (value, derivative) of the two faces normal to a
    ts += 4.0 * F[a];
    fsum += 2.0 * F[a];
  }
  cell += N * 2.0 * (m[0] + m[1] + m[2]);                     // gradient
  cell += N * (tri ? 156.0 : 14.0) + (kappa ? N : 0.0);      // pointwise flux and mass
  cell += N * 2.0 * (m[0] + m[1] + m[2]);                     // transposed derivative
  const double ninner = (double)(nface - nbface);
  const double per_face = (fsum / 6.0);                        // mean points per face
  const double pt_inner = tri ? 250.0 + 8.0 * (m[0] + m[1] + m[2]) / 3.0 : 16.0;
  const double pt_bdry = tri ? 130.0 + 4.0 * (m[0] + m[1] + m[2]) / 3.0 : 10.0;
  const double face = (ninner * pt_inner + (double)nbface * pt_bdry) * per_face;
  const double back = N * 16.0 + 2.0 * (S2 * m[2] + S1 * m[1] + P * m[0]);
  flops[0] = cell * (double)ncell;
  flops[1] = face;
  flops[2] = back * (double)ncell;
  bytes[0] = es * (double)ncell * (P + ts + N + (kappa ? N : 0.0));
  bytes[1] = es * (double)ncell * (2.0 * ts + (kappa ? fsum / 2.0 : 0.0));
  bytes[2] = es * (double)ncell * (N + ts + P);
}
