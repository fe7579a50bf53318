// Per-quadrature-point geometry of trilinear cells (each cell T is the image of the
// reference cube under the trilinear map mu_T through its eight vertices, Sec. 2.1).
//
// Volume, per Gauss point: G = W detJ J^-1 J^-T (6 symmetric entries) and the mass
// weight c W detJ, so that int kappa grad u . grad v + c u v becomes
// grad_ref v^T (kappa G) grad_ref u + (c W detJ) u v.
// Faces, per face Gauss point: with n_vec the area vector (unit normal times the surface
// element) oriented from T- to T+ (outward on boundary faces), b = W J^-1 n_vec for each
// side, so that n . grad u ds = b . grad_ref u, and pw = gamma_F W |n_vec|.
#include "dg_scalar_kernels.cuh"
#include "dg_geo_device.cuh"

namespace {

using namespace dgg;

struct Rule {
  double s[DG_MAXM], w[DG_MAXM];
};

template <typename T>
__global__ void k_geo_vol(int m, int nx, int ny, int64_t ncell, const double *__restrict__ verts, double c,
                          Rule rule, T *__restrict__ gvol) {
  const int m3 = m * m * m;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell * m3) return;
  const int64_t cell = i / m3;
  const int q = (int)(i - cell * m3);
  const int q0 = q % m, q1 = (q / m) % m, q2 = q / (m * m);
  double V[8][3], J[3][3], A[3][3];
  cell_corners(verts, nx, ny, cell, V);
  trilinear_jacobian(V, rule.s[q0], rule.s[q1], rule.s[q2], J);
  const double det = adjugate(J, A);
  const double W = rule.w[q0] * rule.w[q1] * rule.w[q2];
  // G = W det J^-1 J^-T = (W / det) adj adj^T
  const double s = W / det;
  double G[6];
  int e = 0;
  for (int r = 0; r < 3; ++r)
    for (int cc = r; cc < 3; ++cc) G[e++] = s * (A[r][0] * A[cc][0] + A[r][1] * A[cc][1] + A[r][2] * A[cc][2]);
  T *out = gvol + cell * 7 * m3 + q;
  for (int k = 0; k < 6; ++k) out[k * m3] = (T)G[k];
  out[6 * m3] = (T)(c * W * det);
}

template <typename T>
__global__ void k_geo_face(int m, const ScalarArgs<T> a, const double *__restrict__ verts,
                           const double *__restrict__ gamma, Rule rule, T *__restrict__ gface) {
  const int m2 = m * m;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nface * m2) return;
  const int64_t f = i / m2;
  const int qf = (int)(i - f * m2);
  const int qs = qf % m, qt = qf / m;
  const dgk::FaceId F = dgk::decode_face(a, f);
  const int ax = F.axis;
  const double W = rule.w[qs] * rule.w[qt];
  double xi[3];
  xi[F.t1] = rule.s[qs];
  xi[F.t2] = rule.s[qt];
  double V[8][3], J[3][3], A[3][3], n[3];
  double out[7] = {0, 0, 0, 0, 0, 0, 0};
  // first side: T- at xi_a = 1, or the single cell of a boundary face
  const bool lower_bnd = F.cm < 0;
  const int64_t c1 = lower_bnd ? F.cp : F.cm;
  xi[ax] = lower_bnd ? 0.0 : 1.0;
  cell_corners(verts, a.nx, a.ny, c1, V);
  trilinear_jacobian(V, xi[0], xi[1], xi[2], J);
  area_vector(J, ax, lower_bnd ? -1 : 1, n);
  double det = adjugate(J, A);
  for (int r = 0; r < 3; ++r) out[r] = W * (A[r][0] * n[0] + A[r][1] * n[1] + A[r][2] * n[2]) / det;
  out[6] = gamma[f] * W * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (F.cm >= 0 && F.cp >= 0) {
    xi[ax] = 0.0;
    cell_corners(verts, a.nx, a.ny, F.cp, V);
    trilinear_jacobian(V, xi[0], xi[1], xi[2], J);
    det = adjugate(J, A);
    for (int r = 0; r < 3; ++r) out[3 + r] = W * (A[r][0] * n[0] + A[r][1] * n[1] + A[r][2] * n[2]) / det;
  }
  T *o = gface + f * 7 * m2 + qf;
  for (int k = 0; k < 7; ++k) o[k * m2] = (T)out[k];
}

// |T| by the Gauss rule, one thread per cell.
__global__ void k_cell_measure(int m, int nx, int ny, int64_t ncell, const double *__restrict__ verts, Rule rule,
                               double *__restrict__ vol) {
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  double V[8][3], J[3][3], A[3][3], s = 0.0;
  cell_corners(verts, nx, ny, cell, V);
  for (int q2 = 0; q2 < m; ++q2)
    for (int q1 = 0; q1 < m; ++q1)
      for (int q0 = 0; q0 < m; ++q0) {
        trilinear_jacobian(V, rule.s[q0], rule.s[q1], rule.s[q2], J);
        s += rule.w[q0] * rule.w[q1] * rule.w[q2] * adjugate(J, A);
      }
  vol[cell] = s;
}

// gamma_F per face: mode 0 alpha k(k+1) n_a; mode 1 alpha k(k+d-1)|F| / min |T|.
__global__ void k_gamma(int m, int k, int mode, double alpha, const ScalarArgs<double> a,
                        const double *__restrict__ verts, const double *__restrict__ vol, Rule rule,
                        double *__restrict__ gamma) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.nface) return;
  const dgk::FaceId F = dgk::decode_face(a, f);
  const int ax = F.axis;
  const int na = ax == 0 ? a.nx : (ax == 1 ? a.ny : a.nz);
  if (mode == 0) {
    gamma[f] = alpha * k * (k + 1) * (double)na;
    return;
  }
  const bool lower_bnd = F.cm < 0;
  const int64_t c1 = lower_bnd ? F.cp : F.cm;
  double V[8][3], J[3][3], n[3], xi[3], area = 0.0;
  cell_corners(verts, a.nx, a.ny, c1, V);
  xi[ax] = lower_bnd ? 0.0 : 1.0;
  for (int qt = 0; qt < m; ++qt)
    for (int qs = 0; qs < m; ++qs) {
      xi[F.t1] = rule.s[qs];
      xi[F.t2] = rule.s[qt];
      trilinear_jacobian(V, xi[0], xi[1], xi[2], J);
      area_vector(J, ax, 1, n);
      area += rule.w[qs] * rule.w[qt] * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    }
  double T = vol[c1];
  if (F.cm >= 0 && F.cp >= 0) T = fmin(T, vol[F.cp]);
  gamma[f] = alpha * k * (k + 2) * area / T;
}

Rule make_rule(int m, const double *s, const double *w) {
  Rule r;
  for (int i = 0; i < DG_MAXM; ++i) {
    r.s[i] = i < m ? s[i] : 0.0;
    r.w[i] = i < m ? w[i] : 0.0;
  }
  return r;
}

}  // namespace

cudaError_t launch_penalty(int m, int k, int pen_mode, double alpha, int nx, int ny, int nz, int64_t nface,
                           const int64_t *face_off, const double *verts, const double *gauss_s,
                           const double *gauss_w, double *gamma_face, double *cell_vol, cudaStream_t s) {
  ScalarArgs<double> a{};
  a.nx = nx; a.ny = ny; a.nz = nz;
  a.ncell = (int64_t)nx * ny * nz;
  a.nface = nface;
  for (int i = 0; i < 4; ++i) a.face_off[i] = face_off[i];
  Rule rule = make_rule(m, gauss_s, gauss_w);
  if (pen_mode == 1) {
    k_cell_measure<<<(unsigned)((a.ncell + 127) / 128), 128, 0, s>>>(m, nx, ny, a.ncell, verts, rule, cell_vol);
  }
  k_gamma<<<(unsigned)((nface + 127) / 128), 128, 0, s>>>(m, k, pen_mode, alpha, a, verts, cell_vol, rule, gamma_face);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_geometry(int m, const ScalarArgs<T> &a, const double *verts, double c, const double *gamma_face,
                            const double *gauss_s, const double *gauss_w, T *gvol, T *gface, cudaStream_t s) {
  Rule rule = make_rule(m, gauss_s, gauss_w);
  const int64_t nv = a.ncell * m * m * m, nf = a.nface * m * m;
  k_geo_vol<T><<<(unsigned)((nv + 127) / 128), 128, 0, s>>>(m, a.nx, a.ny, a.ncell, verts, c, rule, gvol);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_geo_face<T><<<(unsigned)((nf + 127) / 128), 128, 0, s>>>(m, a, verts, gamma_face, rule, gface);
  return cudaGetLastError();
}

template cudaError_t launch_geometry<double>(int, const ScalarArgs<double> &, const double *, double, const double *,
                                             const double *, const double *, double *, double *, cudaStream_t);
template cudaError_t launch_geometry<float>(int, const ScalarArgs<float> &, const double *, double, const double *,
                                            const double *, const double *, float *, float *, cudaStream_t);
