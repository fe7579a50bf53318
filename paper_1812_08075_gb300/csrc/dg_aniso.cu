// Scalar SIPG apply with anisotropic degrees (Sec. 2.1's vector k = (k_0, k_1, k_2)) on
// affine (axis-parallel) cells: the three-kernel structure of the isotropic apply with
// run-time extents. Direction a has p_a = k_a + 1 GLL basis points and m_a = p_a Gauss
// points, so every stage of a cell's sum factorisation holds p_0 p_1 p_2 values.
//   k_an_cell: interpolation to the Gauss points one direction at a time (Algorithm 1),
//     the traces of the six faces (face normal to a: m_t1 x m_t2 points), the gradient,
//     the pointwise flux with the diagonal affine metric, and the transposed derivative.
//   k_an_face: per face, the jump, average flux and penalty from both sides' traces
//     (Eq. diffreac_weak), written as each side's (value, normal-derivative) residuals.
//   k_an_back: lifting of the face residuals and the transposed interpolation.
// Per cell the traces and face residuals are [6 faces][2][m_t1 m_t2] with per-face offsets.
#include <string.h>

#include "dg_scalar_kernels.cuh"

namespace dgn {

using dgk::decode_face;
using dgk::FaceId;

template <typename T>
struct AnTab {
  int p[3], m[3];
  int toff[7];  // offset of face lf's (value, derivative) pair in a cell's trace block; toff[6] = size
  T interp[3][DG_MAXM * DG_MAXP];  // [a][q * p_a + j]
  T dcol[3][DG_MAXM * DG_MAXM];    // [a][q * m_a + r]
  T e0[3][DG_MAXM], e1[3][DG_MAXM], d0[3][DG_MAXM], d1[3][DG_MAXM], w[3][DG_MAXM];
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

template <typename T>
__global__ void __launch_bounds__(256) k_an_cell(const ScalarArgs<T> a, const AnTab<T> *__restrict__ gtab,
                                                 const T *__restrict__ x, T *__restrict__ rvol,
                                                 T *__restrict__ traces, int cpb, int64_t sdof, int64_t srv,
                                                 int64_t str) {
  __shared__ AnTab<T> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_tab(tb, gtab);
  __syncthreads();
  const int *m = tb.m, *p = tb.p;
  const int N = m[0] * m[1] * m[2], TS = tb.toff[6];
  T *A = reinterpret_cast<T *>(smem_raw), *B = A + cpb * N, *U = B + cpb * N;
  T *F0 = U + cpb * N, *F1 = F0 + cpb * N, *F2 = F1 + cpb * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  x += blockIdx.y * sdof;
  rvol += blockIdx.y * srv;
  traces += blockIdx.y * str;
  for (int i = tid; i < nc * N; i += nt) A[i] = x[c0 * N + i];
  __syncthreads();
  // interpolation: x-sweep A -> B [q0 + m0 (j1 + p1 j2)], y-sweep B -> A, z-sweep A -> U
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, r = i - c * N, q0 = r % m[0], j12 = r / m[0];
    const T *src = A + c * N + j12 * p[0];
    T s = T(0);
    for (int j = 0; j < p[0]; ++j) s = fma(tb.interp[0][q0 * p[0] + j], src[j], s);
    B[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, r = i - c * N, q0 = r % m[0], q1 = (r / m[0]) % m[1], j2 = r / (m[0] * m[1]);
    const T *src = B + c * N + q0 + m[0] * p[1] * j2;
    T s = T(0);
    for (int j = 0; j < p[1]; ++j) s = fma(tb.interp[1][q1 * p[1] + j], src[j * m[0]], s);
    A[i] = s;
  }
  __syncthreads();
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
  // gradient and pointwise flux (affine: diagonal metric), mass term
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, q = i - c * N;
    const int q0 = q % m[0], q1 = (q / m[0]) % m[1], q2 = q / (m[0] * m[1]);
    const T *u = U + c * N;
    T g0 = T(0), g1 = T(0), g2 = T(0);
    for (int k = 0; k < m[0]; ++k) g0 = fma(tb.dcol[0][q0 * m[0] + k], u[k + m[0] * (q1 + m[1] * q2)], g0);
    for (int k = 0; k < m[1]; ++k) g1 = fma(tb.dcol[1][q1 * m[1] + k], u[q0 + m[0] * (k + m[1] * q2)], g1);
    for (int k = 0; k < m[2]; ++k) g2 = fma(tb.dcol[2][q2 * m[2] + k], u[q0 + m[0] * (q1 + m[1] * k)], g2);
    const T W = tb.w[0][q0] * tb.w[1][q1] * tb.w[2][q2];
    F0[i] = W * a.vol_g[0] * g0;
    F1[i] = W * a.vol_g[1] * g1;
    F2[i] = W * a.vol_g[2] * g2;
    B[i] = W * a.vol_m * u[q];
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

template <typename T>
__global__ void __launch_bounds__(256) k_an_face(const ScalarArgs<T> a, const AnTab<T> *__restrict__ gtab,
                                                 const T *__restrict__ traces, T *__restrict__ fres, int fpb,
                                                 int64_t str) {
  __shared__ AnTab<T> tb;
  stage_tab(tb, gtab);
  __syncthreads();
  const int *m = tb.m;
  const int TS = tb.toff[6];
  traces += blockIdx.y * str;
  fres += blockIdx.y * str;
  const int64_t f0 = (int64_t)blockIdx.x * fpb;
  const int nf = (int)min((int64_t)fpb, a.nface - f0);
  const int mf = DG_MAXM * DG_MAXM;  // points per face, at most
  const T sc = a.sc, ss = a.ss, half = T(0.5);
  for (int i = threadIdx.x; i < nf * mf; i += blockDim.x) {
    const int lfc = i / mf, qf = i - lfc * mf;
    const FaceId Fc = decode_face(a, f0 + lfc);
    const int ax = Fc.axis;
    int t1, t2;
    tangential(ax, t1, t2);
    const int F = m[t1] * m[t2];
    if (qf >= F) continue;
    const int qs = qf % m[t1], qt = qf / m[t1];
    const T W = tb.w[t1][qs] * tb.w[t2][qt];
    const T bW = W * a.face_b[ax], pw = W * a.face_pw[ax];
    if (Fc.cm >= 0 && Fc.cp >= 0) {
      const int64_t om = Fc.cm * TS + tb.toff[2 * ax + 1], op = Fc.cp * TS + tb.toff[2 * ax];
      const T um = traces[om + qf], dm = traces[om + F + qf];
      const T up = traces[op + qf], dp = traces[op + F + qf];
      const T J = um - up;
      const T v = fma(sc, half * bW * (dm + dp), pw * J);
      const T rn = ss * half * J * bW;
      fres[om + qf] = v;
      fres[om + F + qf] = rn;
      fres[op + qf] = -v;
      fres[op + F + qf] = rn;
    } else {
      const int side = Fc.cm >= 0 ? 1 : 0;
      const int64_t cb = side ? Fc.cm : Fc.cp;
      const int lf = 2 * ax + side;
      const int64_t ob = cb * TS + tb.toff[lf];
      T rv = T(0), rn = T(0);
      if ((a.dmask >> lf) & 1u) {
        const T uo = traces[ob + qf], dno = traces[ob + F + qf];
        const T b = side ? bW : -bW;
        rv = fma(sc, b * dno, pw * uo);
        rn = ss * uo * b;
      }
      fres[ob + qf] = rv;
      fres[ob + F + qf] = rn;
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
  const int N = m[0] * m[1] * m[2], TS = tb.toff[6];
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
  // transposed interpolation: z (A -> B [q0 + m0 (q1 + m1 j2)]), y (B -> A), x (A -> y)
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, r = i - c * N, q01 = r % (m[0] * m[1]), j2 = r / (m[0] * m[1]);
    const T *src = A + c * N + q01;
    T s = T(0);
    for (int q = 0; q < m[2]; ++q) s = fma(tb.interp[2][q * p[2] + j2], src[q * m[0] * m[1]], s);
    B[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, r = i - c * N, q0 = r % m[0], j1 = (r / m[0]) % p[1], j2 = r / (m[0] * p[1]);
    const T *src = B + c * N + q0 + m[0] * m[1] * j2;
    T s = T(0);
    for (int q = 0; q < m[1]; ++q) s = fma(tb.interp[1][q * p[1] + j1], src[q * m[0]], s);
    A[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < nc * N; i += nt) {
    const int c = i / N, r = i - c * N, j0 = r % p[0], j12 = r / p[0];
    const T *src = A + c * N + j12 * m[0];
    T s = T(0);
    for (int q = 0; q < m[0]; ++q) s = fma(tb.interp[0][q * p[0] + j0], src[q], s);
    y[(c0 + c) * N + r] = s;
  }
}

inline int threads_for(int work) {
  const int t = ((work + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}

}  // namespace dgn

// Host side: tables of the three directions (each direction's own 1D tables) and the
// trace offsets. tab_out: device buffer of sizeof(AnTab<T>) bytes.
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
    if (h.m != h.p) return -1;
    t.p[a] = h.p;
    t.m[a] = h.m;
    for (int i = 0; i < h.m * h.p; ++i) t.interp[a][i] = (T)h.interp[i];
    for (int i = 0; i < h.m * h.m; ++i) t.dcol[a][i] = (T)h.dcol[i];
    for (int i = 0; i < h.m; ++i) {
      t.e0[a][i] = (T)h.e0[i]; t.e1[a][i] = (T)h.e1[i];
      t.d0[a][i] = (T)h.d0[i]; t.d1[a][i] = (T)h.d1[i];
      t.w[a][i] = (T)h.gauss_w[i];
    }
  }
  int off = 0;
  for (int lf = 0; lf < 6; ++lf) {
    int t1, t2;
    dgn::tangential(lf >> 1, t1, t2);
    t.toff[lf] = off;
    off += 2 * t.m[t1] * t.m[t2];
  }
  t.toff[6] = off;
  *trace_size = off;
  return 0;
}

template <typename T>
cudaError_t launch_aniso_apply(const ScalarArgs<T> &a, const void *dtab, int npts, int trace_size, const T *x, T *y,
                               T *rvol, T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str,
                               int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev) {
  using namespace dgn;
  const AnTab<T> *tab = reinterpret_cast<const AnTab<T> *>(dtab);
  cudaError_t e;
  const size_t smc = (size_t)cpb * 6 * npts * sizeof(T), smb = (size_t)cpb * 2 * npts * sizeof(T);
  if (smc > 48 * 1024 &&
      (e = cudaFuncSetAttribute(k_an_cell<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc)) != cudaSuccess)
    return e;
  if (smb > 48 * 1024 &&
      (e = cudaFuncSetAttribute(k_an_back<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb)) != cudaSuccess)
    return e;
  const dim3 gc((unsigned)((a.ncell + cpb - 1) / cpb), nrhs), gf((unsigned)((a.nface + fpb - 1) / fpb), nrhs);
  if (ev) cudaEventRecord(ev[0], s);
  k_an_cell<T><<<gc, threads_for(cpb * npts), smc, s>>>(a, tab, x, rvol, traces, cpb, sdof, srv, str);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  k_an_face<T><<<gf, threads_for(fpb * DG_MAXM * DG_MAXM), 0, s>>>(a, tab, traces, fres, fpb, str);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  k_an_back<T><<<gc, threads_for(cpb * npts), smb, s>>>(a, tab, rvol, fres, y, cpb, sdof, srv, str);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  return cudaSuccess;
}

template size_t aniso_tab_bytes<double>();
template size_t aniso_tab_bytes<float>();
template int aniso_tables<double>(const HostTables[3], void *, int *);
template int aniso_tables<float>(const HostTables[3], void *, int *);
template cudaError_t launch_aniso_apply<double>(const ScalarArgs<double> &, const void *, int, int, const double *,
                                                double *, double *, double *, double *, int, int64_t, int64_t,
                                                int64_t, int, int, cudaStream_t, const cudaEvent_t *);
template cudaError_t launch_aniso_apply<float>(const ScalarArgs<float> &, const void *, int, int, const float *,
                                               float *, float *, float *, float *, int, int64_t, int64_t, int64_t,
                                               int, int, cudaStream_t, const cudaEvent_t *);

// Exact operation counts of the three kernels (FMA = 2) and their algorithmic bytes.
void aniso_work_model(const int kax[3], int64_t ncell, int64_t nface, int64_t nbface, double flops[3],
                      double bytes[3], int es) {
  const double p0 = kax[0] + 1, p1 = kax[1] + 1, p2 = kax[2] + 1, N = p0 * p1 * p2;
  const double F[3] = {p1 * p2, p0 * p2, p0 * p1};  // face points normal to each axis
  const double pa[3] = {p0, p1, p2};
  double cell = N * ((2 * p0 - 1) + (2 * p1 - 1) + (2 * p2 - 1));  // interpolation
  double ts = 0.0;
  for (int a = 0; a < 3; ++a) {
    cell += 2 * 2 * F[a] * (2 * pa[a] - 1);  // traces of the two faces normal to a
    ts += 4 * F[a];
  }
  cell += N * ((2 * p0 - 1) + (2 * p1 - 1) + (2 * p2 - 1) + 3 * 2 + 3);  // gradient, flux, mass
  cell += N * 2 * (p0 + p1 + p2);                                       // transposed derivative
  double face = 0.0;
  const double ninner = (double)(nface - nbface);
  for (int a = 0; a < 3; ++a) face += F[a];
  face = (ninner * 12.0 + (double)nbface * 8.0) * (face / 3.0);
  const double back = N * 24.0 + N * ((2 * p2 - 1) + (2 * p1 - 1) + (2 * p0 - 1));
  flops[0] = cell * (double)ncell;
  flops[1] = face;
  flops[2] = back * (double)ncell;
  bytes[0] = es * (double)ncell * (2 * N + ts);
  bytes[1] = es * (double)ncell * 2 * ts;
  bytes[2] = es * (double)ncell * (2 * N + ts);
}
