// Data terms of the diffusion-reaction residual (Eq. diffreac_weak, Sec. 5.2) moved to
// the right-hand side: F(v) = (f, v) + theta (g, n.kappa grad v)_{Gamma_D}
// + gamma_F (g, v)_{Gamma_D}, so that the residual of Sec. 2.1 is r(u) = A u - F.
//
// Assembled like the second half of an apply: k_rhs_vol writes the Gauss-point residual
// W detJ f, k_rhs_face writes each cell face's (value, normal-derivative) residual pair
// (the Dirichlet data terms on Dirichlet boundary faces, zero elsewhere), and k_back lifts
// the face pairs and applies the transposed interpolation. Trilinear geometry is
// recomputed from the vertex coordinates.
#include "dg_geo_device.cuh"
#include "dg_scalar_kernels.cuh"

namespace dgr {

using namespace dgk;

template <int M, typename T, int GEO>
__global__ void k_rhs_vol(const ScalarArgs<T> a, const T *__restrict__ f, T *__restrict__ rvol) {
  constexpr int M3 = M * M * M;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.ncell * M3) return;
  const int64_t cell = i / M3;
  const int q = (int)(i - cell * M3);
  const int q0 = q % M, q1 = (q / M) % M, q2 = q / (M * M);
  const T *w = a.tab->w;
  const T W = w[q0] * w[q1] * w[q2];
  T wdet;
  if (GEO == GEO_AFFINE) {
    wdet = W / T((double)a.nx * a.ny * a.nz);
  } else {
    double V[8][3], J[3][3], A[3][3];
    dgg::cell_corners(a.verts, a.nx, a.ny, cell, V);
    const T *s = a.tab->s;
    dgg::trilinear_jacobian(V, s[q0], s[q1], s[q2], J);
    wdet = W * (T)dgg::adjugate(J, A);
  }
  rvol[i] = f ? wdet * f[i] : T(0);
}

template <int M, typename T, int GEO, bool KAPPA>
__global__ void __launch_bounds__(256) k_rhs_face(const ScalarArgs<T> a, const T theta, const T *__restrict__ g,
                                                  T *__restrict__ fres, int fpb) {
  constexpr int M2 = M * M;
  __shared__ T sd[M * M];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *SR = reinterpret_cast<T *>(smem_raw);  // [face][3][M2]: Rv, Rt1, Rt2
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < M2; i += nt) sd[i] = a.tab->dcol[i];
  __syncthreads();
  const int64_t f0 = (int64_t)blockIdx.x * fpb;
  const int nf = (int)min((int64_t)fpb, a.nface - f0);
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const int64_t f = f0 + lfc;
    const FaceId F = decode_face(a, f);
    const int ax = F.axis, t1 = F.t1, t2 = F.t2;
    const int qs = qf % M, qt = qf / M;
    T *R = SR + lfc * 3 * M2;
    if (F.cm >= 0 && F.cp >= 0) {
      fres[tr_idx<M>(F.cm, 2 * ax + 1, 0, qf)] = T(0);
      fres[tr_idx<M>(F.cm, 2 * ax + 1, 1, qf)] = T(0);
      fres[tr_idx<M>(F.cp, 2 * ax, 0, qf)] = T(0);
      fres[tr_idx<M>(F.cp, 2 * ax, 1, qf)] = T(0);
      R[qf] = R[M2 + qf] = R[2 * M2 + qf] = T(0);
      continue;
    }
    const int side = F.cm >= 0 ? 1 : 0;
    const int64_t cb = side ? F.cm : F.cp;
    const int lf = 2 * ax + side;
    T Rv = T(0), Rn = T(0), Rt1 = T(0), Rt2 = T(0);
    if (g && ((a.dmask >> lf) & 1u)) {
      const T *w = a.tab->w;
      const T W = w[qs] * w[qt];
      const T gv = g[(cb * 6 + lf) * M2 + qf];
      const T kb = KAPPA ? a.kappa_face[(cb * 6 + lf) * M2 + qf] : T(1);
      T b[3] = {T(0), T(0), T(0)}, pw;
      if (GEO == GEO_AFFINE) {
        b[ax] = (side ? W : -W) * a.face_b[ax];
        pw = W * a.face_pw[ax];
      } else {
        double V[8][3], J[3][3], A[3][3], n[3], xi[3];
        const T *s = a.tab->s;
        xi[ax] = side ? 1.0 : 0.0;
        xi[t1] = s[qs];
        xi[t2] = s[qt];
        dgg::cell_corners(a.verts, a.nx, a.ny, cb, V);
        dgg::trilinear_jacobian(V, xi[0], xi[1], xi[2], J);
        dgg::area_vector(J, ax, side ? 1 : -1, n);
        const double det = dgg::adjugate(J, A);
        for (int r = 0; r < 3; ++r) b[r] = (T)(W * (A[r][0] * n[0] + A[r][1] * n[1] + A[r][2] * n[2]) / det);
        pw = (T)(a.gamma_face[f] * W * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]));
      }
      const T tg = theta * kb * gv;
      Rv = pw * gv;
      Rn = tg * b[ax];
      Rt1 = tg * b[t1];
      Rt2 = tg * b[t2];
    }
    fres[tr_idx<M>(cb, lf, 1, qf)] = Rn;
    R[qf] = Rv;
    R[M2 + qf] = Rt1;
    R[2 * M2 + qf] = Rt2;
  }
  __syncthreads();
  for (int i = tid; i < nf * M2; i += nt) {
    const int lfc = i / M2, qf = i - lfc * M2;
    const FaceId F = decode_face(a, f0 + lfc);
    if (F.cm >= 0 && F.cp >= 0) continue;
    const int ax = F.axis, side = F.cm >= 0 ? 1 : 0;
    const int qs = qf % M, qt = qf / M;
    const T *R = SR + lfc * 3 * M2;
    T v = R[qf];
#pragma unroll
    for (int r = 0; r < M; ++r) {
      v = fma(sd[r * M + qs], R[M2 + r + qt * M], v);
      v = fma(sd[r * M + qt], R[2 * M2 + qs + r * M], v);
    }
    fres[tr_idx<M>(side ? F.cm : F.cp, 2 * ax + side, 0, qf)] = v;
  }
}

template <int P, typename T, int GEO, bool KAPPA>
cudaError_t run(const ScalarArgs<T> &a, T theta, const T *f, const T *g, T *F, T *rvol, T *fres, int cpb, int fpb,
                cudaStream_t s) {
  constexpr int M = P, M2 = M * M, M3 = M * M * M;
  const int64_t nv = a.ncell * M3;
  k_rhs_vol<M, T, GEO><<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(a, f, rvol);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int thr = fpb * M2 < 64 ? 64 : (fpb * M2 > 256 ? 256 : ((fpb * M2 + 31) / 32) * 32);
  k_rhs_face<M, T, GEO, KAPPA><<<(unsigned)((a.nface + fpb - 1) / fpb), thr, (size_t)fpb * 3 * M2 * sizeof(T), s>>>(
      a, theta, g, fres, fpb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t sm = back_smem_bytes<P, M, T>(cpb);
  if (sm > 48 * 1024 &&
      (e = cudaFuncSetAttribute(k_back<P, M, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  const int tb = cpb * M3 < 64 ? 64 : (cpb * M3 > 256 ? 256 : ((cpb * M3 + 31) / 32) * 32);
  k_back<P, M, T><<<dim3((unsigned)((a.ncell + cpb - 1) / cpb), 1), tb, sm, s>>>(a, rvol, fres, F, cpb, 0, 0, 0);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t run_p(int geo, bool kappa, const ScalarArgs<T> &a, T theta, const T *f, const T *g, T *F, T *rvol,
                  T *fres, int cpb, int fpb, cudaStream_t s) {
  if (geo == GEO_AFFINE) {
    if (kappa) return run<P, T, GEO_AFFINE, true>(a, theta, f, g, F, rvol, fres, cpb, fpb, s);
    return run<P, T, GEO_AFFINE, false>(a, theta, f, g, F, rvol, fres, cpb, fpb, s);
  }
  if (kappa) return run<P, T, GEO_RECOMPUTE, true>(a, theta, f, g, F, rvol, fres, cpb, fpb, s);
  return run<P, T, GEO_RECOMPUTE, false>(a, theta, f, g, F, rvol, fres, cpb, fpb, s);
}

}  // namespace dgr

template <typename T>
cudaError_t launch_rhs(int p, int geo, bool kappa, const ScalarArgs<T> &a, T theta, const T *f, const T *g, T *F,
                       T *rvol, T *fres, int cpb, int fpb, cudaStream_t s) {
  switch (p) {
    case 2: return dgr::run_p<2, T>(geo, kappa, a, theta, f, g, F, rvol, fres, cpb, fpb, s);
    case 3: return dgr::run_p<3, T>(geo, kappa, a, theta, f, g, F, rvol, fres, cpb, fpb, s);
    case 4: return dgr::run_p<4, T>(geo, kappa, a, theta, f, g, F, rvol, fres, cpb, fpb, s);
    case 5: return dgr::run_p<5, T>(geo, kappa, a, theta, f, g, F, rvol, fres, cpb, fpb, s);
    case 6: return dgr::run_p<6, T>(geo, kappa, a, theta, f, g, F, rvol, fres, cpb, fpb, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_rhs<double>(int, int, bool, const ScalarArgs<double> &, double, const double *,
                                        const double *, double *, double *, double *, int, int, cudaStream_t);
template cudaError_t launch_rhs<float>(int, int, bool, const ScalarArgs<float> &, float, const float *, const float *,
                                       float *, float *, float *, int, int, cudaStream_t);
