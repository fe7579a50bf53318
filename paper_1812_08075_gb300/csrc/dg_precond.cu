// Cell-block Jacobi preconditioner z_c = A_cc^-1 r_c by fast diagonalisation, for the
// scalar SIPG operator on affine (axis-parallel) cells with kappa = 1 and theta = -1.
//
// On such a cell the diagonal block of A (Eq. diffreac_weak restricted to test and trial
// functions of one cell: its volume terms and its own side of its six faces) is a
// Kronecker sum of one-dimensional matrices (Sec. 2.2's tensor structure):
//   A_cc = A_z (x) M (x) M + M (x) A_y (x) M + M (x) M (x) A_x,
// with M the 1D mass matrix of the GLL basis under the Gauss rule and A_d the 1D
// stiffness of axis d plus the cell's own terms of its two faces normal to d (half flux
// weight on interior faces, full weight on Dirichlet faces, nothing on Neumann faces),
// the mass term folded into A_x. With the generalized eigenvectors A_d S_d = M S_d L_d,
// S_d^T M S_d = I, the inverse is
//   A_cc^-1 = (S_z (x) S_y (x) S_x) (L_z (+) L_y (+) L_x)^-1 (S_z (x) S_y (x) S_x)^T,
// applied by sum factorisation: three transposed sweeps, a pointwise division, three
// sweeps. A_d depends on the cell's position along d (interior, first, last, only cell),
// so each axis has four (S, L) pairs, computed once on the host in FP64.
#include <math.h>
#include <string.h>

#include <vector>

#include "dg_df64.cuh"
#include "dg_internal.h"

namespace {

// Cyclic Jacobi eigenvalue method for a symmetric n x n matrix a (row-major, destroyed):
// a = q diag(l) q^T (Golub & Van Loan, Matrix Computations, Sec. 8.5).
void jacobi_eigen(int n, double *a, double *q, double *l) {
  for (int i = 0; i < n * n; ++i) q[i] = 0.0;
  for (int i = 0; i < n; ++i) q[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int r = p + 1; r < n; ++r) {
        const double apr = a[p * n + r];
        if (apr == 0.0) continue;
        const double theta = (a[r * n + r] - a[p * n + p]) / (2.0 * apr);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, r
          const double akp = a[k * n + p], akr = a[k * n + r];
          a[k * n + p] = c * akp - s * akr;
          a[k * n + r] = s * akp + c * akr;
        }
        for (int k = 0; k < n; ++k) {  // rows p, r
          const double apk = a[p * n + k], ark = a[r * n + k];
          a[p * n + k] = c * apk - s * ark;
          a[r * n + k] = s * apk + c * ark;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = q[k * n + p], qkr = q[k * n + r];
          q[k * n + p] = c * qkp - s * qkr;
          q[k * n + r] = s * qkp + c * qkr;
        }
      }
  }
  for (int i = 0; i < n; ++i) l[i] = a[i * n + i];
}

// S (column eigenvectors, row-major [i][col]) and L with A S = M S diag(L), S^T M S = I,
// for symmetric A and symmetric positive definite M: M = C C^T (Cholesky), eigenvectors
// Q of C^-1 A C^-T, S = C^-T Q. Returns false if M is not positive definite.
bool generalized_eigen(int n, const double *A, const double *M, double *S, double *L) {
  std::vector<double> C(n * n, 0.0), X(n * n), B(n * n), Q(n * n);
  for (int j = 0; j < n; ++j) {
    double d = M[j * n + j];
    for (int k = 0; k < j; ++k) d -= C[j * n + k] * C[j * n + k];
    if (!(d > 0.0)) return false;
    C[j * n + j] = sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double v = M[i * n + j];
      for (int k = 0; k < j; ++k) v -= C[i * n + k] * C[j * n + k];
      C[i * n + j] = v / C[j * n + j];
    }
  }
  // X = C^-1 A (forward substitution on each column), B = X C^-T = (C^-1 X^T)^T
  for (int col = 0; col < n; ++col)
    for (int i = 0; i < n; ++i) {
      double v = A[i * n + col];
      for (int k = 0; k < i; ++k) v -= C[i * n + k] * X[k * n + col];
      X[i * n + col] = v / C[i * n + i];
    }
  for (int row = 0; row < n; ++row)  // B[row][i] = (C^-1 X^T)[i][row]
    for (int i = 0; i < n; ++i) {
      double v = X[row * n + i];
      for (int k = 0; k < i; ++k) v -= C[i * n + k] * B[row * n + k];
      B[row * n + i] = v / C[i * n + i];
    }
  for (int i = 0; i < n; ++i)  // symmetrise the rounding
    for (int j = i + 1; j < n; ++j) B[i * n + j] = B[j * n + i] = 0.5 * (B[i * n + j] + B[j * n + i]);
  jacobi_eigen(n, B.data(), Q.data(), L);
  // S = C^-T Q (back substitution on each column)
  for (int col = 0; col < n; ++col)
    for (int i = n - 1; i >= 0; --i) {
      double v = Q[i * n + col];
      for (int k = i + 1; k < n; ++k) v -= C[k * n + i] * S[k * n + col];
      S[i * n + col] = v / C[i * n + i];
    }
  return true;
}

enum { FACE_INTERIOR = 0, FACE_DIRICHLET = 1, FACE_NONE = 2 };

template <int P, typename T>
struct BJTab {
  T S[3][4][P * P];  // [axis][position][i * P + col]
};

// z = A_cc^-1 r, one thread per tensor line of a group of cpb consecutive cells; the
// blocks loop over the groups. dinv[(16 px + 4 py + pz) P^3 + point] holds
// 1 / (Lx + Ly + Lz) for the cell's positions. Partials of r.z per block go to
// partial[rhs * stride + block] (FP64) when non-NULL.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_block_jacobi(const BJTab<P, T> tb, const T *__restrict__ dinv,
                                                      const T *__restrict__ r, T *__restrict__ z, int nx, int ny,
                                                      int nz, int64_t ncell, int cpb, int64_t sdof, double *partial,
                                                      int stride) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ T sS[3 * 4 * P2];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *A = reinterpret_cast<T *>(smem_raw);  // [cell][P3]
  T *B = A + cpb * P3;
  const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int pos = 0; pos < 4; ++pos)
      for (int i = tid; i < P2; i += nt) sS[(d * 4 + pos) * P2 + i] = tb.S[d][pos][i];
  auto position = [](int c, int n) { return n == 1 ? 3 : (c == 0 ? 1 : (c == n - 1 ? 2 : 0)); };
  // this thread's line (the block has at least cpb P^2 threads): cell ci, line (l1, l2)
  const bool has_line = tid < cpb * P2;
  const int ci = tid / P2, l = tid - ci * P2, l1 = l % P, l2 = l / P;
  const int64_t ngroups = (ncell + cpb - 1) / cpb;
  double dot = 0.0;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t c0 = grp * cpb;
    const int nc = (int)min((int64_t)cpb, ncell - c0);
    const T *rr = r + blockIdx.y * sdof + c0 * P3;
    T *zz = z + blockIdx.y * sdof + c0 * P3;
    const bool act = has_line && ci < nc;
    int px = 0, py = 0, pz = 0;
    if (act) {
      const int64_t cell = c0 + ci;
      const int64_t cyz = cell / nx;
      px = position((int)(cell - cyz * nx), nx);
      py = position((int)(cyz % ny), ny);
      pz = position((int)(cyz / ny), nz);
    }
    __syncthreads();  // tables staged / previous group's A consumed
    for (int i = tid; i < nc * P3; i += nt) A[i] = rr[i];
    __syncthreads();
    auto sweep = [&](const T *in, T *out, int axis, bool transposed, bool scale) {
      if (act) {
        const int pos = axis == 0 ? px : (axis == 1 ? py : pz);
        const T *S = sS + (axis * 4 + pos) * P2;
        int base, st;
        if (axis == 0) { base = P * l1 + P2 * l2; st = 1; }
        else if (axis == 1) { base = l1 + P2 * l2; st = P; }
        else { base = l1 + P * l2; st = P2; }
        const T *v = in + ci * P3 + base;
        T *o = out + ci * P3 + base;
        const T *di = dinv + (16 * px + 4 * py + pz) * P3 + base;  // the z sweep: point (l1, l2, i)
        T vin[P];
#pragma unroll
        for (int j = 0; j < P; ++j) vin[j] = v[j * st];
#pragma unroll
        for (int i = 0; i < P; ++i) {
          T s = T(0);
#pragma unroll
          for (int j = 0; j < P; ++j) s = fma(transposed ? S[j * P + i] : S[i * P + j], vin[j], s);
          if (scale) s *= __ldg(di + i * st);
          o[i * st] = s;
        }
      }
      __syncthreads();
    };
    sweep(A, B, 0, true, false);
    sweep(B, A, 1, true, false);
    sweep(A, B, 2, true, true);
    sweep(B, A, 2, false, false);
    sweep(A, B, 1, false, false);
    sweep(B, A, 0, false, false);
    for (int i = tid; i < nc * P3; i += nt) {
      const T v = A[i];
      zz[i] = v;
      dot = fma((double)rr[i], (double)v, dot);
    }
  }
  if (partial) {
    __shared__ double part[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
    if ((tid & 31) == 0) part[tid >> 5] = dot;
    __syncthreads();
    if (tid < 32) {
      double w = tid < (nt >> 5) ? part[tid] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
      if (tid == 0) partial[blockIdx.y * stride + blockIdx.x] = w;
    }
  }
}

// The same for FP32 and k <= 2 with one thread per cell and the cell in registers: a block of 128
// threads takes 128 consecutive cells (r and z staged through shared memory for coalesced
// rows), and each axis sweep is instantiated for the four cell positions with the table
// entries as constant-bank operands. The 32 consecutive cells of a warp share their y and z
// positions unless a row is shorter than a warp, so only the x sweeps diverge, and only in
// warps holding a first or last cell of a row.
template <int P, typename T, int AX, bool TR>
__device__ __forceinline__ void bj_sweep_pos(const BJTab<P, T> &tb, int pos, const T *in, T *out) {
  constexpr int P2 = P * P;
  auto run = [&](const T *S) {
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b) {
        // line (a, b) over the two other axes in increasing order
        auto idx = [&](int i) { return AX == 0 ? i + P * a + P2 * b : (AX == 1 ? a + P * i + P2 * b : a + P * b + P2 * i); };
#pragma unroll
        for (int i = 0; i < P; ++i) {
          T s = T(0);
#pragma unroll
          for (int j = 0; j < P; ++j) s = fma(TR ? S[j * P + i] : S[i * P + j], in[idx(j)], s);
          out[idx(i)] = s;
        }
      }
  };
  switch (pos) {
    case 0: run(tb.S[AX][0]); break;
    case 1: run(tb.S[AX][1]); break;
    case 2: run(tb.S[AX][2]); break;
    default: run(tb.S[AX][3]); break;
  }
}

// The per-cell kernel also runs fused into the vector updates of preconditioned CG: the
// block inverse is local to a cell, so it can be applied where r is produced and where
// the direction is formed instead of in a pass of its own over r and z.
//   BJ_APPLY:     z = A_cc^-1 r, partials of r.z.
//   BJ_UPDATE:    r -= alpha Ap in place, z = A_cc^-1 r in registers (not stored), and
//                 the partials of r.z and r.r.
//   BJ_DIRECTION: z = A_cc^-1 r again, then x += alpha p and p = z + beta p with the old p
//                 (p only while the right-hand side is active).
// alpha, beta and the active flags are per right-hand side (device). A right-hand side
// with alpha = 0 is left unchanged and contributes zero partials. V4: the rows of x, r,
// Ap, p move as 16-byte vectors (FP32, sdof a multiple of 4, 16-byte aligned buffers);
// the element order of every sum is the same with and without V4.
template <typename T>
struct BJFuse {
  const double *alpha, *beta;
  const int *active;
  const T *Ap;
  T *x, *p;
  double *prr;  // r.r partials (BJ_UPDATE)
};

template <int P, typename T, int MODE, bool V4>
__global__ void __launch_bounds__(128) k_block_jacobi_cell(const BJTab<P, T> tb, const T *__restrict__ dinv,
                                                           const T *__restrict__ r_in, T *__restrict__ rz_out,
                                                           const BJFuse<T> fu, int nx, int ny, int nz, int64_t ncell,
                                                           int64_t sdof, double *partial, int stride) {
  constexpr int P3 = P * P * P, sX = P3 | 1, NB = 128;
  __shared__ __align__(16) T st[NB * sX];
  auto position = [](int c, int n) { return n == 1 ? 3 : (c == 0 ? 1 : (c == n - 1 ? 2 : 0)); };
  auto sidx = [](int i) { const int c = i / P3; return c * sX + (i - c * P3); };  // chunk element -> row slot
  const int tid = threadIdx.x, rhs = blockIdx.y;
  const T *src = MODE == BJ_UPDATE ? rz_out : r_in;  // BJ_UPDATE updates r in place (r_in unused)
  const int64_t nchunks = (ncell + NB - 1) / NB;
  const T a = MODE == BJ_APPLY ? T(0) : (T)fu.alpha[rhs];
  const bool act = MODE == BJ_DIRECTION ? fu.active[rhs] != 0 : true;
  DotAcc<T> acc_rz, acc_rr;  // r.z and r.r at FP64-class accuracy (double-float for FP32)
  const bool work = MODE == BJ_APPLY || a != T(0);
  for (int64_t ch = blockIdx.x; work && ch < nchunks; ch += gridDim.x) {
    const int64_t c0 = ch * NB;
    const int nc = (int)min((int64_t)NB, ncell - c0), ne = nc * P3, n4 = V4 ? ne / 4 : 0;
    const int64_t off = rhs * sdof + c0 * P3;
    __syncthreads();  // the previous chunk's rows were read out
    if (act) {  // stage r (after r -= alpha Ap for BJ_UPDATE)
      if constexpr (V4) {
        for (int i = tid; i < n4; i += NB) {
          float4 v = ((const float4 *)(src + off))[i];
          if constexpr (MODE == BJ_UPDATE) {
            const float4 q = ((const float4 *)(fu.Ap + off))[i];
            v = make_float4(fmaf(-a, q.x, v.x), fmaf(-a, q.y, v.y), fmaf(-a, q.z, v.z), fmaf(-a, q.w, v.w));
            ((float4 *)(rz_out + off))[i] = v;
          }
          st[sidx(4 * i)] = v.x;
          st[sidx(4 * i + 1)] = v.y;
          st[sidx(4 * i + 2)] = v.z;
          st[sidx(4 * i + 3)] = v.w;
        }
      }
      for (int i = 4 * n4 + tid; i < ne; i += NB) {
        T v = src[off + i];
        if constexpr (MODE == BJ_UPDATE) {
          v = fma(-a, fu.Ap[off + i], v);
          rz_out[off + i] = v;
        }
        st[sidx(i)] = v;
      }
      __syncthreads();
      if (tid < nc) {
        const int64_t cell = c0 + tid, cyz = cell / nx;
        const int px = position((int)(cell - cyz * nx), nx), py = position((int)(cyz % ny), ny),
                  pz = position((int)(cyz / ny), nz);
        T u[P3], v[P3];
#pragma unroll
        for (int i = 0; i < P3; ++i) u[i] = st[tid * sX + i];
        bj_sweep_pos<P, T, 0, true>(tb, px, u, v);
        bj_sweep_pos<P, T, 1, true>(tb, py, v, u);
        bj_sweep_pos<P, T, 2, true>(tb, pz, u, v);
        const T *di = dinv + (16 * px + 4 * py + pz) * P3;
#pragma unroll
        for (int i = 0; i < P3; ++i) v[i] *= __ldg(di + i);
        bj_sweep_pos<P, T, 2, false>(tb, pz, v, u);
        bj_sweep_pos<P, T, 1, false>(tb, py, u, v);
        bj_sweep_pos<P, T, 0, false>(tb, px, v, u);
#pragma unroll
        for (int i = 0; i < P3; ++i) {
          const T ri = st[tid * sX + i];
          acc_rz.add(ri, u[i]);
          if constexpr (MODE == BJ_UPDATE) acc_rr.add(ri, ri);
          if constexpr (MODE != BJ_UPDATE) st[tid * sX + i] = u[i];
        }
      }
      __syncthreads();
    }
    if constexpr (MODE == BJ_APPLY) {
      if constexpr (V4) {
        for (int i = tid; i < n4; i += NB)
          ((float4 *)(rz_out + off))[i] =
              make_float4(st[sidx(4 * i)], st[sidx(4 * i + 1)], st[sidx(4 * i + 2)], st[sidx(4 * i + 3)]);
      }
      for (int i = 4 * n4 + tid; i < ne; i += NB) rz_out[off + i] = st[sidx(i)];
    } else if constexpr (MODE == BJ_DIRECTION) {  // x += alpha p, p = z + beta p (old p)
      const T b = act ? (T)fu.beta[rhs] : T(0);
      if constexpr (V4) {
        for (int i = tid; i < n4; i += NB) {
          const float4 q = ((const float4 *)(fu.p + off))[i];
          float4 *X = (float4 *)(fu.x + off) + i;
          const float4 xv = *X;
          *X = make_float4(fmaf(a, q.x, xv.x), fmaf(a, q.y, xv.y), fmaf(a, q.z, xv.z), fmaf(a, q.w, xv.w));
          if (act)
            ((float4 *)(fu.p + off))[i] = make_float4(fmaf(b, q.x, st[sidx(4 * i)]), fmaf(b, q.y, st[sidx(4 * i + 1)]),
                                                      fmaf(b, q.z, st[sidx(4 * i + 2)]), fmaf(b, q.w, st[sidx(4 * i + 3)]));
        }
      }
      for (int i = 4 * n4 + tid; i < ne; i += NB) {
        const T q = fu.p[off + i];
        fu.x[off + i] = fma(a, q, fu.x[off + i]);
        if (act) fu.p[off + i] = fma(b, q, st[sidx(i)]);
      }
    }
  }
  if (MODE != BJ_DIRECTION && partial) {
    double dot = acc_rz.value(), dot2 = acc_rr.value();
    __shared__ double part[2][NB / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dot += __shfl_down_sync(0xffffffffu, dot, o);
      dot2 += __shfl_down_sync(0xffffffffu, dot2, o);
    }
    if ((tid & 31) == 0) { part[0][tid >> 5] = dot; part[1][tid >> 5] = dot2; }
    __syncthreads();
    if (tid == 0) {
      double w = 0.0, w2 = 0.0;
      for (int i = 0; i < NB / 32; ++i) { w += part[0][i]; w2 += part[1][i]; }
      partial[rhs * stride + blockIdx.x] = w;
      if (MODE == BJ_UPDATE) fu.prr[rhs * stride + blockIdx.x] = w2;
    }
  }
}

template <int P, typename T>
BJTab<P, T> device_tab(const double *tab) {
  BJTab<P, T> tb;
  for (int d = 0; d < 3; ++d)
    for (int pos = 0; pos < 4; ++pos) {
      const double *src = tab + (d * 4 + pos) * (P * P + P);
      for (int i = 0; i < P * P; ++i) tb.S[d][pos][i] = (T)src[i];
    }
  return tb;
}

// one wave of 16 blocks of 128 threads per SM over the right-hand sides, at most `stride`
// blocks per right-hand side when partials are written
inline int64_t cell_blocks(int64_t ncell, int nrhs, bool partial, int stride) {
  const int64_t nchunks = (ncell + 127) / 128;
  const int64_t wave = 16 * (int64_t)dg_device_sms();
  int64_t nb = wave / nrhs > 0 ? wave / nrhs : 1;
  if (partial && nb > stride) nb = stride;
  return nb > nchunks ? nchunks : nb;
}

template <typename T>
bool vec4_ok(int64_t sdof, const void *a, const void *b, const void *c, const void *d) {
  auto al = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
  return sizeof(T) == 4 && sdof % 4 == 0 && al(a) && al(b) && al(c) && al(d);
}

template <int P, typename T>
cudaError_t run_bj(const double *tab, const T *dinv, int nx, int ny, int nz, int64_t ncell, const T *r, T *z, int nrhs,
                   int64_t sdof, double *partial, int stride, int *blocks, cudaStream_t s) {
  const BJTab<P, T> tb = device_tab<P, T>(tab);
  if constexpr (P <= 3 && sizeof(T) == 4) {  // one thread per cell (FP64 stays on the lines: fewer registers, no divergence)
    const int64_t nb = cell_blocks(ncell, nrhs, partial != nullptr, stride);
    if (blocks) *blocks = (int)nb;
    const BJFuse<T> none{};
    const dim3 g((unsigned)nb, nrhs);
    if (vec4_ok<T>(sdof, r, z, z, z))
      k_block_jacobi_cell<P, T, BJ_APPLY, true><<<g, 128, 0, s>>>(tb, dinv, r, z, none, nx, ny, nz, ncell, sdof, partial,
                                                                  stride);
    else
      k_block_jacobi_cell<P, T, BJ_APPLY, false><<<g, 128, 0, s>>>(tb, dinv, r, z, none, nx, ny, nz, ncell, sdof,
                                                                   partial, stride);
    return cudaGetLastError();
  }
  const int cpb = 256 / (P * P) > 0 ? 256 / (P * P) : 1;
  const int threads = ((cpb * P * P + 31) / 32) * 32;
  const size_t sm = 2 * (size_t)cpb * P * P * P * sizeof(T);
  // one wave of 8 blocks per SM over the right-hand sides, at most `stride` per rhs
  const int64_t ngroups = (ncell + cpb - 1) / cpb;
  const int64_t wave = 8 * (int64_t)dg_device_sms();
  int64_t nb = wave / nrhs > 0 ? wave / nrhs : 1;
  if (partial && nb > stride) nb = stride;
  if (nb > ngroups) nb = ngroups;
  if (blocks) *blocks = (int)nb;
  k_block_jacobi<P, T><<<dim3((unsigned)nb, nrhs), threads, sm, s>>>(tb, dinv, r, z, nx, ny, nz, ncell, cpb, sdof,
                                                                      partial, stride);
  return cudaGetLastError();
}

template <int P, int MODE>
cudaError_t run_bj_fused(const double *tab, const float *dinv, const dg_operator *op, float *r, const BJFuse<float> &fu,
                         int nrhs, double *prz, int stride, int *blocks, cudaStream_t s) {
  const BJTab<P, float> tb = device_tab<P, float>(tab);
  const int64_t sdof = op->ndofs, nb = cell_blocks(op->ncell, nrhs, true, stride);
  if (blocks) *blocks = (int)nb;
  const dim3 g((unsigned)nb, nrhs);
  const bool v4 = MODE == BJ_UPDATE ? vec4_ok<float>(sdof, r, fu.Ap, r, r) : vec4_ok<float>(sdof, r, fu.x, fu.p, r);
  const float *rin = MODE == BJ_UPDATE ? nullptr : r;
  float *rout = MODE == BJ_UPDATE ? r : nullptr;
  if (v4)
    k_block_jacobi_cell<P, float, MODE, true><<<g, 128, 0, s>>>(tb, dinv, rin, rout, fu, op->nx, op->ny, op->nz,
                                                                op->ncell, sdof, prz, stride);
  else
    k_block_jacobi_cell<P, float, MODE, false><<<g, 128, 0, s>>>(tb, dinv, rin, rout, fu, op->nx, op->ny, op->nz,
                                                                 op->ncell, sdof, prz, stride);
  return cudaGetLastError();
}

}  // namespace

// 1D factors and their generalized eigen-decompositions for the operator (host, FP64):
// tab[(axis * 4 + position) * (P^2 + P) + ...] = S (row-major), then L.
int block_jacobi_tables(const dg_operator *op, std::vector<double> &tab) {
  const HostTables &h = op->ht;
  const int P = h.p, m = h.m;
  if (op->problem != DG_SCALAR || op->geo != GEO_AFFINE || op->kappa_vol || m != P || op->theta != -1.0) return -1;
  std::vector<double> M(P * P, 0.0), K(P * P, 0.0), G(m * P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j)
      for (int q = 0; q < m; ++q) M[i * P + j] += h.gauss_w[q] * h.interp[q * P + i] * h.interp[q * P + j];
  for (int q = 0; q < m; ++q)  // derivative of the GLL basis at the Gauss points
    for (int j = 0; j < P; ++j)
      for (int r = 0; r < m; ++r) G[q * P + j] += h.dcol[q * m + r] * h.interp[r * P + j];
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j)
      for (int q = 0; q < m; ++q) K[i * P + j] += h.gauss_w[q] * G[q * P + i] * G[q * P + j];
  const double hh[3] = {1.0 / op->nx, 1.0 / op->ny, 1.0 / op->nz};
  const double V = hh[0] * hh[1] * hh[2];
  const double sc = -1.0, ss = op->theta;  // forward face coefficients
  tab.assign(12 * (P * P + P), 0.0);
  std::vector<double> A(P * P);
  for (int d = 0; d < 3; ++d) {
    const double vg = V / (hh[d] * hh[d]), fb = V / (hh[d] * hh[d]), fpw = op->gamma_axis[d] * V / hh[d];
    const int lo_bnd = (op->dmask >> (2 * d)) & 1u ? FACE_DIRICHLET : FACE_NONE;
    const int hi_bnd = (op->dmask >> (2 * d + 1)) & 1u ? FACE_DIRICHLET : FACE_NONE;
    for (int pos = 0; pos < 4; ++pos) {
      const int lo = (pos == 1 || pos == 3) ? lo_bnd : FACE_INTERIOR;
      const int hi = (pos == 2 || pos == 3) ? hi_bnd : FACE_INTERIOR;
      for (int i = 0; i < P * P; ++i) A[i] = vg * K[i] + (d == 0 ? op->c * V * M[i] : 0.0);
      // own side of the face at xi = 0 (GLL basis: value e_0 = delta_0, derivative gd0)
      if (lo != FACE_NONE) {
        const double hb = (lo == FACE_INTERIOR ? 0.5 : 1.0) * fb;
        for (int j = 0; j < P; ++j) {
          A[0 * P + j] += -sc * hb * h.gd0[j];
          A[j * P + 0] += -ss * hb * h.gd0[j];
        }
        A[0] += fpw;
      }
      if (hi != FACE_NONE) {  // face at xi = 1 (value e_{P-1}, derivative gd1)
        const double hb = (hi == FACE_INTERIOR ? 0.5 : 1.0) * fb;
        for (int j = 0; j < P; ++j) {
          A[(P - 1) * P + j] += sc * hb * h.gd1[j];
          A[j * P + (P - 1)] += ss * hb * h.gd1[j];
        }
        A[(P - 1) * P + (P - 1)] += fpw;
      }
      double *dst = tab.data() + (d * 4 + pos) * (P * P + P);
      if (!generalized_eigen(P, A.data(), M.data(), dst, dst + P * P)) return -2;
    }
  }
  return 0;
}

// 1 / (Lx[i0] + Ly[i1] + Lz[i2]) for the 64 combinations of cell positions (px, py, pz),
// [(16 px + 4 py + pz) P^3 + i0 + P (i1 + P i2)], from the tables above.
void block_jacobi_inverse_sums(int P, const std::vector<double> &tab, std::vector<double> &dinv) {
  const int P3 = P * P * P;
  dinv.assign(64 * P3, 0.0);
  auto L = [&](int d, int pos) { return tab.data() + (d * 4 + pos) * (P * P + P) + P * P; };
  for (int px = 0; px < 4; ++px)
    for (int py = 0; py < 4; ++py)
      for (int pz = 0; pz < 4; ++pz)
        for (int i2 = 0; i2 < P; ++i2)
          for (int i1 = 0; i1 < P; ++i1)
            for (int i0 = 0; i0 < P; ++i0) {
              const double sum = L(0, px)[i0] + L(1, py)[i1] + L(2, pz)[i2];
              dinv[(16 * px + 4 * py + pz) * P3 + i0 + P * (i1 + P * i2)] = sum != 0.0 ? 1.0 / sum : 0.0;
            }
}

template <typename T>
cudaError_t launch_block_jacobi(const dg_operator *op, const double *tab, const T *dinv, const T *r, T *z, int nrhs,
                                double *partial, int stride, int *blocks, cudaStream_t s) {
  const int64_t sdof = op->ndofs;
  switch (op->p) {
#define DG_BJ_CASE(PP)                                                                                            \
  case PP:                                                                                                        \
    return run_bj<PP, T>(tab, dinv, op->nx, op->ny, op->nz, op->ncell, r, z, nrhs, sdof, partial, stride, blocks, s);
    DG_BJ_CASE(2)
    DG_BJ_CASE(3)
    DG_BJ_CASE(4)
    DG_BJ_CASE(5)
    DG_BJ_CASE(6)
#undef DG_BJ_CASE
    default: return cudaErrorInvalidValue;
  }
}

bool block_jacobi_fusable(const dg_operator *op) { return op->precision == DG_FP32 && op->p <= 3; }

cudaError_t launch_block_jacobi_fused(const dg_operator *op, const double *tab, const float *dinv, int mode, float *r,
                                      const float *Ap, float *x, float *p, const double *alpha, const double *beta,
                                      const int *active, int nrhs, double *prz, double *prr, int stride, int *blocks,
                                      cudaStream_t s) {
  if (!block_jacobi_fusable(op) || (mode != BJ_UPDATE && mode != BJ_DIRECTION)) return cudaErrorInvalidValue;
  const BJFuse<float> fu{alpha, beta, active, Ap, x, p, prr};
  if (mode == BJ_UPDATE)
    return op->p == 2 ? run_bj_fused<2, BJ_UPDATE>(tab, dinv, op, r, fu, nrhs, prz, stride, blocks, s)
                      : run_bj_fused<3, BJ_UPDATE>(tab, dinv, op, r, fu, nrhs, prz, stride, blocks, s);
  return op->p == 2 ? run_bj_fused<2, BJ_DIRECTION>(tab, dinv, op, r, fu, nrhs, nullptr, stride, blocks, s)
                    : run_bj_fused<3, BJ_DIRECTION>(tab, dinv, op, r, fu, nrhs, nullptr, stride, blocks, s);
}

template cudaError_t launch_block_jacobi<double>(const dg_operator *, const double *, const double *, const double *,
                                                 double *, int, double *, int, int *, cudaStream_t);
template cudaError_t launch_block_jacobi<float>(const dg_operator *, const double *, const float *, const float *,
                                                float *, int, double *, int, int *, cudaStream_t);
