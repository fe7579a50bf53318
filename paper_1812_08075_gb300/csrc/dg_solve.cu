// Krylov solves on top of the matrix-free apply: batched conjugate gradients for up to
// 16 right-hand sides at once (each right-hand side its own independent CG with its
// own scalars), and FP64 iterative refinement around an FP32 inner CG.
//
// CG on A d = r: dot products accumulate in FP64 whatever the vector precision; the
// per-right-hand-side scalars (alpha, beta, r.z, convergence flag) live on the device,
// so a chunk of iterations runs without host round trips and is captured once into a
// CUDA graph and replayed. A right-hand side that has converged gets alpha = 0 and stops
// changing while the others continue. Refinement keeps the residual b - A x, the update
// x += d and all inner products in FP64 and uses the FP32 operator only inside CG.
#include <math.h>
#include <string.h>

#include <vector>

#include <algorithm>

#include "dg_df64.cuh"
#include "dg_internal.h"

namespace {

struct Scalars {  // device, one entry per right-hand side
  double rz[16], rz_new[16], pAp[16], rr[16], alpha[16], beta[16], tol2[16], bb[16];
  int active[16], iters[16], breakdown[16];
};

constexpr int kThreads = 256;
// Row stride of the per-block partial sums: room for the largest grid of the vector
// kernels (16 blocks per SM, up to 256 SMs). The grid is fixed per vector size and device,
// so the reduction order is too.
constexpr int kMaxBlocks = 4096;

// Scalars followed by per-block partial sums [16 rhs][kMaxBlocks] of the reductions.
struct Workspace {
  Scalars S;
  double partial[16 * kMaxBlocks];
  double partial2[16 * kMaxBlocks];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v written to partial[rhs * kMaxBlocks + block] (no atomics: the final sum
// in k_reduce runs in a fixed order, so reductions are bitwise reproducible).
__device__ __forceinline__ void block_partial(double v, double *partial) {
  __shared__ double part[kThreads / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    w = warp_sum(w);
    if (threadIdx.x == 0) partial[blockIdx.y * kMaxBlocks + blockIdx.x] = w;
  }
  __syncthreads();
}

// Two block sums at once (same fixed order as block_partial).
__device__ __forceinline__ void block_partial2(double v, double w, double *pa, double *pb) {
  __shared__ double part[2][kThreads / 32];
  v = warp_sum(v);
  w = warp_sum(w);
  if ((threadIdx.x & 31) == 0) { part[0][threadIdx.x >> 5] = v; part[1][threadIdx.x >> 5] = w; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = threadIdx.x < (blockDim.x >> 5);
    double a = in ? part[0][threadIdx.x] : 0.0, b = in ? part[1][threadIdx.x] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
      pa[blockIdx.y * kMaxBlocks + blockIdx.x] = a;
      pb[blockIdx.y * kMaxBlocks + blockIdx.x] = b;
    }
  }
  __syncthreads();
}

// out[rhs] = sum of the nblocks partials of rhs (one block per rhs, fixed order)
__global__ void k_reduce(const double *__restrict__ partial, double *out, int nblocks) {
  __shared__ double sh[kThreads];
  const int rhs = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partial[rhs * kMaxBlocks + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[rhs] = sh[0];
}

// Vector kernels come in two forms. The scalar form (any T) accumulates every product
// in FP64. The float4 form (V4, FP32 vectors whose length is a multiple of 4 and whose
// buffers are 16-byte aligned) moves four elements per access and accumulates the
// products in double-float on the FP32 pipes (DotAcc<float>: each product's rounding error
// kept exactly, FP64-class accuracy), since one FP64 operation per element would bound
// these kernels by the FP64 pipe of this part instead of by memory.
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {  // a x + y
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

template <typename T, bool V4>
__global__ void k_residual(const T *__restrict__ b, const T *__restrict__ Ax, T *__restrict__ r, int64_t n) {
  const int64_t off = (int64_t)blockIdx.y * n;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  if constexpr (V4) {
    const float4 *B = (const float4 *)(b + off), *A = (const float4 *)(Ax + off);
    float4 *R = (float4 *)(r + off);
    for (int64_t i = i0; i < n / 4; i += st) R[i] = axpy4(-1.0f, A[i], B[i]);
  } else {
    for (int64_t i = i0; i < n; i += st) r[off + i] = b[off + i] - Ax[off + i];
  }
}

// partials of u . v per rhs (FP64 accumulation); k_reduce finishes the sum
template <typename T, bool V4>
__global__ void k_dot(const T *__restrict__ u, const T *__restrict__ v, double *partial, int64_t n) {
  const int64_t off = (int64_t)blockIdx.y * n;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  double s = 0.0;
  if constexpr (V4) {
    const float4 *U = (const float4 *)(u + off), *V = (const float4 *)(v + off);
    DotAcc<float> acc;
    for (int64_t i = i0; i < n / 4; i += st) acc.add4(U[i], V[i]);
    s = acc.value();
  } else {
    for (int64_t i = i0; i < n; i += st) s = fma((double)u[off + i], (double)v[off + i], s);
  }
  block_partial(s, partial);
}

// Start of CG: z = D^-1 r (dinv NULL: z = r), p = z, partials of r.z and r.r.
template <typename T, bool V4>
__global__ void k_init_dir(const T *__restrict__ r, T *__restrict__ p, const T *__restrict__ dinv, double *prz,
                           double *prr, int64_t n) {
  const int64_t off = (int64_t)blockIdx.y * n;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  double s = 0.0, t = 0.0;
  if constexpr (V4) {
    const float4 *R = (const float4 *)(r + off), *D = (const float4 *)dinv;
    float4 *Pv = (float4 *)(p + off);
    DotAcc<float> as, at;
    for (int64_t i = i0; i < n / 4; i += st) {
      const float4 v = R[i];
      const float4 z = dinv ? mul4(D[i], v) : v;
      Pv[i] = z;
      as.add4(v, z);
      at.add4(v, v);
    }
    s = as.value();
    t = at.value();
  } else {
    for (int64_t i = i0; i < n; i += st) {
      const T v = r[off + i];
      const T z = dinv ? dinv[i] * v : v;
      p[off + i] = z;
      s = fma((double)v, (double)z, s);
      t = fma((double)v, (double)v, t);
    }
  }
  block_partial2(s, t, prz, prr);
}

// r.z (z = D^-1 r, dinv NULL: z = r) and r.r without writing a direction (reliable updates).
template <typename T>
__global__ void k_refresh(const T *__restrict__ r, const T *__restrict__ dinv, double *prz, double *prr, int64_t n) {
  const int64_t off = (int64_t)blockIdx.y * n;
  double s = 0.0, t = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = r[off + i];
    s = fma((double)v, (double)(dinv ? dinv[i] * v : v), s);
    t = fma((double)v, (double)v, t);
  }
  block_partial2(s, t, prz, prr);
}

// Per rhs: reactivate (1) or stop (0) from a host flag array after a reliable update.
__global__ void k_set_active(Scalars *S, const int *flags, int nrhs) {
  const int r = threadIdx.x;
  if (r < nrhs) S->active[r] = flags[r];
}

__global__ void k_init_scalars(Scalars *S, int nrhs, double rtol) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  S->tol2[r] = rtol * rtol * S->bb[r];
  S->active[r] = S->rr[r] > S->tol2[r] ? 1 : 0;
  S->pAp[r] = 0.0;
  S->iters[r] = 0;
  S->breakdown[r] = 0;
}

// Restart from a recomputed residual (rz = r.r already reduced): iteration counts kept.
__global__ void k_restart_scalars(Scalars *S, int nrhs) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  S->active[r] = S->rr[r] > S->tol2[r] ? 1 : 0;
  S->pAp[r] = 0.0;
}

__global__ void k_alpha(Scalars *S, int nrhs) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  double a = 0.0;
  if (S->active[r]) {
    if (S->pAp[r] > 0.0) {
      a = S->rz[r] / S->pAp[r];
    } else {  // A not positive definite in this direction (or roundoff): stop this rhs
      S->active[r] = 0;
      S->breakdown[r] = 1;
    }
  }
  S->alpha[r] = a;
}

// x += alpha p, r -= alpha Ap, and the partials of r.z (z = D^-1 r) and r.r
template <typename T, bool V4>
__global__ void k_update(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ Ap,
                         const T *__restrict__ dinv, const Scalars *S, double *prz, double *prr, int64_t n) {
  const int rhs = blockIdx.y;
  const int64_t off = (int64_t)rhs * n;
  const double ad = S->alpha[rhs];
  double s = 0.0, t = 0.0;
  if constexpr (V4) {
    if (ad != 0.0) {
      const float a = (float)ad;
      float4 *X = (float4 *)(x + off), *R = (float4 *)(r + off);
      const float4 *Pv = (const float4 *)(p + off), *A = (const float4 *)(Ap + off), *D = (const float4 *)dinv;
      DotAcc<float> as, at;
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 4; i += (int64_t)gridDim.x * blockDim.x) {
        X[i] = axpy4(a, Pv[i], X[i]);
        const float4 v = axpy4(-a, A[i], R[i]);
        R[i] = v;
        if (dinv) {
          as.add4(v, mul4(D[i], v));
          at.add4(v, v);
        } else {
          as.add4(v, v);
        }
      }
      s = as.value();
      t = at.value();
    }
    block_partial2(s, dinv ? t : s, prz, prr);
    return;
  }
  if (ad != 0.0) {
    const T a = (T)ad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      x[off + i] = fma(a, p[off + i], x[off + i]);
      const T v = fma(-a, Ap[off + i], r[off + i]);
      r[off + i] = v;
      if (dinv) {
        s = fma((double)v, (double)(dinv[i] * v), s);
        t = fma((double)v, (double)v, t);
      } else {  // r.z = r.r: one FP64 accumulation per element (FP64 is scarce on this part)
        s = fma((double)v, (double)v, s);
      }
    }
  }
  block_partial2(s, dinv ? t : s, prz, prr);
}

__global__ void k_beta(Scalars *S, int nrhs) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  if (S->active[r]) {
    S->iters[r] += 1;
    S->beta[r] = S->rz_new[r] / S->rz[r];
    S->rz[r] = S->rz_new[r];
    if (S->rr[r] <= S->tol2[r]) S->active[r] = 0;
  } else {
    S->beta[r] = 0.0;
  }
}

template <typename T, bool V4>
__global__ void k_direction(T *__restrict__ p, const T *__restrict__ r, const T *__restrict__ dinv, const Scalars *S,
                            int64_t n) {
  const int rhs = blockIdx.y;
  if (!S->active[rhs]) return;
  const int64_t off = (int64_t)rhs * n;
  const T b = (T)S->beta[rhs];
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  if constexpr (V4) {
    float4 *Pv = (float4 *)(p + off);
    const float4 *R = (const float4 *)(r + off), *D = (const float4 *)dinv;
    for (int64_t i = i0; i < n / 4; i += st) Pv[i] = axpy4(b, Pv[i], dinv ? mul4(D[i], R[i]) : R[i]);
  } else {
    for (int64_t i = i0; i < n; i += st) p[off + i] = fma(b, p[off + i], dinv ? dinv[i] * r[off + i] : r[off + i]);
  }
}

// Unit vectors of one colour (cells whose coordinate parities give `color`) at local DOF j.
template <typename T>
__global__ void k_unit_color(T *__restrict__ e, int64_t ncell, int P3, int nx, int ny, int color, int j) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncell * P3; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = i / P3;
    const int jj = (int)(i - cell * P3);
    const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((int64_t)nx * ny));
    const int col = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
    e[i] = (col == color && jj == j) ? T(1) : T(0);
  }
}

// diag[cell][j] = y[cell][j] for the cells of `color` (optionally inverted)
template <typename T>
__global__ void k_take_color(const T *__restrict__ y, T *__restrict__ diag, int64_t ncell, int P3, int nx, int ny,
                             int color, int j, int invert) {
  for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell; cell += (int64_t)gridDim.x * blockDim.x) {
    const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((int64_t)nx * ny));
    const int col = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
    if (col == color) {
      const T d = y[cell * P3 + j];
      diag[cell * P3 + j] = invert ? T(1) / d : d;
    }
  }
}

__global__ void k_zero_scalars(Scalars *S) {
  double *d = reinterpret_cast<double *>(S);
  for (int i = threadIdx.x; i < 8 * 16; i += blockDim.x) d[i] = 0.0;
}

// x64 += (double) d32
__global__ void k_add_correction(double *__restrict__ x, const float *__restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

unsigned grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  const int64_t cap = std::min<int64_t>(16 * (int64_t)dg_device_sms(), kMaxBlocks);
  return (unsigned)(g > cap ? cap : (g < 1 ? 1 : g));
}

// Blocks per right-hand side of the reducing vector kernels: one wave of 8 blocks per SM
// over all right-hand sides, so every thread streams many elements before the block's
// FP64 reduction tree (FP64 add throughput is scarce on this part; a reduction per few
// elements would cost more than the vector traffic itself).
unsigned grid_vec(int64_t n, int nrhs) {
  const int64_t wave = std::min<int64_t>(8 * (int64_t)dg_device_sms(), kMaxBlocks);
  int64_t g = (n + kThreads - 1) / kThreads;
  const int64_t cap = wave / nrhs > 1 ? wave / nrhs : 1;
  return (unsigned)(g > cap ? cap : (g < 1 ? 1 : g));
}

#define SCK(call)                                          \
  do {                                                     \
    if ((call) != cudaSuccess) return dg_record_error(DG_ERR_CUDA); \
  } while (0)

void drop_graph(dg_operator *op) {
  if (op->sv_graph) cudaGraphExecDestroy((cudaGraphExec_t)op->sv_graph);
  op->sv_graph = nullptr;
  op->sv_graph_key = nullptr;
}

// Workspace in op: vectors r, p, Ap (and d) of the operator's precision, max_rhs each.
dg_status ensure_workspace(dg_operator *op, size_t es) {
  const size_t need = 4 * (size_t)op->max_rhs * op->ndofs * es;
  if (op->sv_vec_bytes < need) {
    drop_graph(op);
    if (op->sv_vec) cudaFree(op->sv_vec);
    op->sv_vec = nullptr;
    op->sv_vec_bytes = 0;
    if (cudaMalloc(&op->sv_vec, need) != cudaSuccess) { cudaGetLastError(); return dg_record_error(DG_ERR_OOM); }
    op->sv_vec_bytes = need;
  }
  if (!op->sv_scal) {
    if (cudaMalloc(&op->sv_scal, sizeof(Workspace)) != cudaSuccess) { cudaGetLastError(); return dg_record_error(DG_ERR_OOM); }
  }
  return DG_OK;
}

// diag(A) (or its inverse) by applying A to unit vectors of one cell colour and one
// local DOF at a time: cells of one colour share no face, so (A e)_i = A_ii on them.
template <typename T>
dg_status diagonal_by_colours(dg_operator *op, T *out, bool invert, cudaStream_t s) {
  const int64_t n = op->ndofs;
  const int P3 = op->p * op->p * op->p;
  T *e = nullptr, *y = nullptr;
  if (cudaMalloc(&e, n * sizeof(T)) != cudaSuccess || cudaMalloc(&y, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    if (e) cudaFree(e);
    return dg_record_error(DG_ERR_OOM);
  }
  dg_status st = DG_OK;
  for (int color = 0; color < 8 && st == DG_OK; ++color)
    for (int j = 0; j < P3 && st == DG_OK; ++j) {
      k_unit_color<T><<<grid_for(n), kThreads, 0, s>>>(e, op->ncell, P3, op->nx, op->ny, color, j);
      st = dg_apply_internal(op, e, y, 1, s, false);
      if (st != DG_OK) break;
      k_take_color<T><<<grid_for(op->ncell), kThreads, 0, s>>>(y, out, op->ncell, P3, op->nx, op->ny, color, j,
                                                                invert ? 1 : 0);
    }
  if (st == DG_OK && cudaStreamSynchronize(s) != cudaSuccess) st = dg_record_error(DG_ERR_CUDA);
  cudaFree(e);
  cudaFree(y);
  return st;
}

dg_status ensure_block_jacobi(dg_operator *op) {
  if (op->aniso) return dg_record_error(DG_ERR_UNSUPPORTED);
  if (!op->bj_tab.empty() && op->d_bjinv) return DG_OK;
  if (block_jacobi_tables(op, op->bj_tab) != 0) {
    op->bj_tab.clear();
    return dg_record_error(DG_ERR_UNSUPPORTED);
  }
  std::vector<double> inv;
  block_jacobi_inverse_sums(op->p, op->bj_tab, inv);
  const size_t es = op->precision == DG_FP64 ? 8 : 4;
  std::vector<float> inv32;
  const void *src = inv.data();
  if (es == 4) {
    inv32.assign(inv.begin(), inv.end());
    src = inv32.data();
  }
  if (cudaMalloc(&op->d_bjinv, inv.size() * es) != cudaSuccess) {
    cudaGetLastError();
    op->d_bjinv = nullptr;
    op->bj_tab.clear();
    return dg_record_error(DG_ERR_OOM);
  }
  if (cudaMemcpy(op->d_bjinv, src, inv.size() * es, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(op->d_bjinv);
    op->d_bjinv = nullptr;
    op->bj_tab.clear();
    return dg_record_error(DG_ERR_CUDA);
  }
  return DG_OK;
}

template <typename T>
dg_status ensure_inverse_diagonal(dg_operator *op, cudaStream_t s) {
  if (op->sv_dinv) return DG_OK;
  if (cudaMalloc(&op->sv_dinv, op->ndofs * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    op->sv_dinv = nullptr;
    return dg_record_error(DG_ERR_OOM);
  }
  dg_status st = diagonal_by_colours<T>(op, (T *)op->sv_dinv, true, s);
  if (st != DG_OK) {
    cudaFree(op->sv_dinv);
    op->sv_dinv = nullptr;
  }
  return st;
}

// The float4 form applies to FP32 vectors of length divisible by 4 whose caller buffers
// (x, b) are 16-byte aligned; the internal vectors then are too.
template <typename T>
bool use_v4(int64_t n, const void *x, const void *b) {
  return sizeof(T) == 4 && n % 4 == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)b & 15) == 0;
}

// Enqueue `iters` CG iterations on x, r, p, Ap (device, [nrhs][n]) with scalars S.
// z (non-NULL): block-Jacobi preconditioning, z = B r computed after the update with the
// r.z partials, and the direction p = z + beta p.
template <typename T, bool V4>
dg_status enqueue_iterations(const dg_operator *op, T *x, T *r, T *p, T *Ap, const T *dinv, T *z, Workspace *W,
                             int nrhs, int iters, cudaStream_t s) {
  const int64_t n = op->ndofs;
  const dim3 g(grid_vec(V4 ? n / 4 : n, nrhs), nrhs);
  Scalars *S = &W->S;
  for (int it = 0; it < iters; ++it) {
    // Ap and p . Ap: in one pass where the operator's kernel forms the dot (FP32 cellwise,
    // two vector passes fewer), else the apply and a dot kernel
    int nbd = 0;
    dg_status st = sizeof(T) == 4 ? dg_apply_dot_internal(op, p, Ap, nrhs, s, W->partial, kMaxBlocks, &nbd)
                                  : DG_ERR_UNSUPPORTED;
    if (st == DG_OK) {
      k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->pAp, nbd);
    } else if (st == DG_ERR_UNSUPPORTED) {
      st = dg_apply_internal(op, p, Ap, nrhs, s, false);
      if (st != DG_OK) return st;
      k_dot<T, V4><<<g, kThreads, 0, s>>>(p, Ap, W->partial, n);
      k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->pAp, g.x);
    } else {
      return st;
    }
    k_alpha<<<1, 32, 0, s>>>(S, nrhs);
    if constexpr (sizeof(T) == 4) {
      if (z && block_jacobi_fusable(op)) {
        // the cell-block inverse inside the two vector passes: r -= alpha Ap with z = B r and
        // the partials of r.z and r.r, then z = B r again with x += alpha p, p = z + beta p
        // (12 vector passes per iteration instead of 15 with z stored)
        int nb = 0;
        const float *bjinv = (const float *)op->d_bjinv;
        SCK(launch_block_jacobi_fused(op, op->bj_tab.data(), bjinv, BJ_UPDATE, r, Ap, x, p, S->alpha, S->beta,
                                      S->active, nrhs, W->partial, W->partial2, kMaxBlocks, &nb, s));
        k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial2, S->rr, nb);
        k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->rz_new, nb);
        k_beta<<<1, 32, 0, s>>>(S, nrhs);
        SCK(launch_block_jacobi_fused(op, op->bj_tab.data(), bjinv, BJ_DIRECTION, r, nullptr, x, p, S->alpha, S->beta,
                                      S->active, nrhs, nullptr, nullptr, kMaxBlocks, nullptr, s));
        continue;
      }
    }
    k_update<T, V4><<<g, kThreads, 0, s>>>(x, r, p, Ap, dinv, S, W->partial, W->partial2, n);
    if (z) {
      k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial2, S->rr, g.x);
      int nb = 0;
      SCK(launch_block_jacobi<T>(op, op->bj_tab.data(), (const T *)op->d_bjinv, r, z, nrhs, W->partial, kMaxBlocks, &nb, s));
      k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->rz_new, nb);
      k_beta<<<1, 32, 0, s>>>(S, nrhs);
      k_direction<T, V4><<<g, kThreads, 0, s>>>(p, z, nullptr, S, n);
      continue;
    }
    k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->rz_new, g.x);
    k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial2, S->rr, g.x);
    k_beta<<<1, 32, 0, s>>>(S, nrhs);
    k_direction<T, V4><<<g, kThreads, 0, s>>>(p, r, dinv, S, n);
  }
  SCK(cudaGetLastError());
  return DG_OK;
}

template <typename T>
void launch_residual(bool v4, dim3 g, cudaStream_t s, const T *b, const T *Ax, T *r, int64_t n) {
  if constexpr (sizeof(T) == 4) {
    if (v4) { k_residual<T, true><<<g, kThreads, 0, s>>>(b, Ax, r, n); return; }
  }
  k_residual<T, false><<<g, kThreads, 0, s>>>(b, Ax, r, n);
}

template <typename T>
void launch_dot(bool v4, dim3 g, cudaStream_t s, const T *u, const T *v, double *partial, int64_t n) {
  if constexpr (sizeof(T) == 4) {
    if (v4) { k_dot<T, true><<<g, kThreads, 0, s>>>(u, v, partial, n); return; }
  }
  k_dot<T, false><<<g, kThreads, 0, s>>>(u, v, partial, n);
}

template <typename T>
void launch_init_dir(bool v4, dim3 g, cudaStream_t s, const T *r, T *p, const T *dinv, double *prz, double *prr,
                     int64_t n) {
  if constexpr (sizeof(T) == 4) {
    if (v4) { k_init_dir<T, true><<<g, kThreads, 0, s>>>(r, p, dinv, prz, prr, n); return; }
  }
  k_init_dir<T, false><<<g, kThreads, 0, s>>>(r, p, dinv, prz, prr, n);
}

template <typename T>
dg_status enqueue(bool v4, const dg_operator *op, T *x, T *r, T *p, T *Ap, const T *dinv, T *z, Workspace *W,
                  int nrhs, int iters, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (v4) return enqueue_iterations<T, true>(op, x, r, p, Ap, dinv, z, W, nrhs, iters, s);
  }
  return enqueue_iterations<T, false>(op, x, r, p, Ap, dinv, z, W, nrhs, iters, s);
}

// Start (or restart) of CG from the residual r: p = z = M^-1 r and the reductions of
// r.z (into S->rz) and r.r (into S->rr).
template <typename T>
dg_status start_directions(const dg_operator *op, bool v4, dim3 g, T *r, T *p, const T *dinv, T *z, Workspace *W,
                           int nrhs, cudaStream_t s) {
  const int64_t n = op->ndofs;
  Scalars *S = &W->S;
  if (z) {
    int nb = 0;
    SCK(launch_block_jacobi<T>(op, op->bj_tab.data(), (const T *)op->d_bjinv, r, z, nrhs, W->partial, kMaxBlocks, &nb, s));
    k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->rz, nb);
    launch_dot<T>(v4, g, s, r, r, W->partial2, n);
    k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial2, S->rr, g.x);
    SCK(cudaMemcpyAsync(p, z, (size_t)nrhs * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return DG_OK;
  }
  launch_init_dir<T>(v4, g, s, r, p, dinv, W->partial, W->partial2, n);
  k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->rz, g.x);
  k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial2, S->rr, g.x);
  return DG_OK;
}

// CG on A x = b for nrhs right-hand sides; x holds the initial guess (x_zero: it is 0
// and b is the initial residual). Fills info[] and returns the status.
// verify: on convergence of the recursive residual, recompute r = b - A x and restart
// (at most 3 times) the right-hand sides whose true residual is still above the target.
template <typename T>
dg_status cg_run(dg_operator *op, const T *b, T *x, int nrhs, const dg_cg_options &o, bool x_zero, bool verify,
                 dg_solve_info *info, cudaStream_t s) {
  const size_t es = sizeof(T);
  dg_status st = ensure_workspace(op, es);
  if (st != DG_OK) return st;
  const int64_t n = op->ndofs;
  T *r = (T *)op->sv_vec, *p = r + op->max_rhs * n, *Ap = p + op->max_rhs * n;
  const T *dinv = nullptr;
  T *z = nullptr;
  if (o.precond == DG_PRECOND_JACOBI) {
    st = ensure_inverse_diagonal<T>(op, s);
    if (st != DG_OK) return st;
    dinv = (const T *)op->sv_dinv;
  } else if (o.precond == DG_PRECOND_BLOCK_JACOBI) {
    st = ensure_block_jacobi(op);
    if (st != DG_OK) return st;
    z = Ap + op->max_rhs * n;
  }
  Workspace *W = (Workspace *)op->sv_scal;
  Scalars *S = &W->S;
  const bool v4 = use_v4<T>(n, x, b);
  const dim3 g(grid_vec(v4 ? n / 4 : n, nrhs), nrhs);
  k_zero_scalars<<<1, 128, 0, s>>>(S);
  if (x_zero) {
    SCK(cudaMemcpyAsync(r, b, (size_t)nrhs * n * es, cudaMemcpyDeviceToDevice, s));
  } else {
    st = dg_apply_internal(op, x, Ap, nrhs, s, false);
    if (st != DG_OK) return st;
    launch_residual<T>(v4, g, s, b, Ap, r, n);
  }
  launch_dot<T>(v4, g, s, b, b, W->partial, n);
  k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->bb, g.x);
  st = start_directions<T>(op, v4, g, r, p, dinv, z, W, nrhs, s);
  if (st != DG_OK) return st;
  k_init_scalars<<<1, 32, 0, s>>>(S, nrhs, o.rtol);
  SCK(cudaGetLastError());
  const int chunk = o.chunk > 0 ? o.chunk : 25;
  // the graph depends on the buffers, nrhs and chunk: rebuild when any of them changes
  void *key = (void *)((uintptr_t)x ^ ((uintptr_t)b << 1) ^ ((uintptr_t)op->kappa_vol << 2) ^
                       ((uintptr_t)op->kappa_face << 3) ^ ((uintptr_t)dinv << 5) ^ ((uintptr_t)z << 7) ^ ((uintptr_t)nrhs << 48) ^
                       ((uintptr_t)chunk << 56));
  cudaStream_t cs = s;
  bool own_stream = false;
  if (o.use_graph && s == 0) {  // the legacy stream cannot be captured
    SCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    own_stream = true;
    SCK(cudaStreamSynchronize(0));
  }
  if (o.use_graph && (op->sv_graph == nullptr || op->sv_graph_key != key)) {
    drop_graph(op);
    const bool prof = op->prof;
    const_cast<dg_operator *>(op)->prof = false;
    cudaGraph_t graph;
    SCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    dg_status est = enqueue<T>(v4, op, x, r, p, Ap, dinv, z, W, nrhs, chunk, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    op->prof = prof;
    if (est != DG_OK) return est;
    if (ce != cudaSuccess) return dg_record_error(DG_ERR_CUDA);
    cudaGraphExec_t exec;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return dg_record_error(DG_ERR_CUDA);
    op->sv_graph = (void *)exec;
    op->sv_graph_key = key;
  }
  Scalars h;
  int done = 0;
  dg_status result = DG_ERR_NOT_CONVERGED;
  for (int restart = 0;; ++restart) {
    result = DG_ERR_NOT_CONVERGED;
    while (done < o.max_iters) {
      if (o.use_graph) {
        SCK(cudaGraphLaunch((cudaGraphExec_t)op->sv_graph, cs));
      } else {
        st = enqueue<T>(v4, op, x, r, p, Ap, dinv, z, W, nrhs, chunk, cs);
        if (st != DG_OK) return st;
      }
      done += chunk;
      SCK(cudaMemcpyAsync(&h, S, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
      SCK(cudaStreamSynchronize(cs));
      int any = 0;
      for (int i = 0; i < nrhs; ++i) any |= h.active[i];
      if (!any) {
        result = DG_OK;
        break;
      }
    }
    if (!verify || result != DG_OK) break;
    st = dg_apply_internal(op, x, Ap, nrhs, cs, false);
    if (st != DG_OK) return st;
    launch_residual<T>(v4, g, cs, b, Ap, r, n);
    st = start_directions<T>(op, v4, g, r, p, dinv, z, W, nrhs, cs);
    if (st != DG_OK) return st;
    k_restart_scalars<<<1, 32, 0, cs>>>(S, nrhs);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(&h, S, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
    SCK(cudaStreamSynchronize(cs));
    int any = 0;
    for (int i = 0; i < nrhs; ++i) any |= h.active[i];
    if (!any || restart >= 3 || done >= o.max_iters) {
      if (any) result = DG_ERR_NOT_CONVERGED;
      break;
    }
  }
  if (result != DG_OK) {
    SCK(cudaMemcpyAsync(&h, S, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
    SCK(cudaStreamSynchronize(cs));
  }
  for (int i = 0; i < nrhs; ++i) {
    info[i].iters = h.iters[i];
    info[i].outer = 0;
    info[i].converged = h.rr[i] <= h.tol2[i] && !h.breakdown[i];
    info[i].breakdown = h.breakdown[i];
    info[i].relres = h.bb[i] > 0 ? sqrt(h.rr[i] / h.bb[i]) : 0.0;
    if (!info[i].converged) result = DG_ERR_NOT_CONVERGED;
  }
  if (own_stream) {
    SCK(cudaStreamSynchronize(cs));
    cudaStreamDestroy(cs);
  }
  return result;
}

// Mixed-precision CG with reliable updates (residual replacement, van der Vorst & Ye):
// FP32 CG iterations with the FP32 operator on A d = r, continued across updates; at an
// update the FP32 correction is added to the FP64 solution, the residual is recomputed in
// FP64 with the FP64 operator and replaces the FP32 one, and the search direction is kept,
// so the Krylov information survives (a refinement step restarts CG instead). An update
// runs when a right-hand side's FP32 residual has fallen by delta since the last one, or
// when the FP32 recursion thinks it has converged; convergence is only declared on the
// FP64 residual. Inner products accumulate in FP64 throughout.
dg_status mixed_cg_run(dg_operator *op64, dg_operator *op32, const double *b, double *x, int nrhs,
                       const dg_cg_options &o, double delta, dg_solve_info *info, cudaStream_t s) {
  const int64_t n = op64->ndofs;
  const size_t nv = (size_t)nrhs * n;
  dg_status st = ensure_workspace(op32, sizeof(float));
  if (st != DG_OK) return st;
  // FP64 residual and A x (op64), FP32 accumulated correction (op32)
  const size_t need64 = nv * 2 * sizeof(double);
  if (op64->sv_aux_bytes < need64) {
    if (op64->sv_aux) cudaFree(op64->sv_aux);
    op64->sv_aux = nullptr;
    op64->sv_aux_bytes = 0;
    if (cudaMalloc(&op64->sv_aux, need64) != cudaSuccess) { cudaGetLastError(); return dg_record_error(DG_ERR_OOM); }
    op64->sv_aux_bytes = need64;
  }
  if (op32->sv_aux_bytes < nv * sizeof(float)) {
    if (op32->sv_aux) cudaFree(op32->sv_aux);
    op32->sv_aux = nullptr;
    op32->sv_aux_bytes = 0;
    if (cudaMalloc(&op32->sv_aux, nv * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return dg_record_error(DG_ERR_OOM); }
    op32->sv_aux_bytes = nv * sizeof(float);
  }
  if (!op64->sv_scal && cudaMalloc(&op64->sv_scal, sizeof(Workspace)) != cudaSuccess) {
    cudaGetLastError();
    return dg_record_error(DG_ERR_OOM);
  }
  double *r64 = (double *)op64->sv_aux, *ax64 = r64 + nv;
  float *r32 = (float *)op32->sv_vec, *p = r32 + op32->max_rhs * n, *Ap = p + op32->max_rhs * n;
  float *x32 = (float *)op32->sv_aux;
  const float *dinv = nullptr;
  float *z = nullptr;
  if (o.precond == DG_PRECOND_JACOBI) {
    if ((st = ensure_inverse_diagonal<float>(op32, s)) != DG_OK) return st;
    dinv = (const float *)op32->sv_dinv;
  } else if (o.precond == DG_PRECOND_BLOCK_JACOBI) {
    if ((st = ensure_block_jacobi(op32)) != DG_OK) return st;
    z = Ap + op32->max_rhs * n;
  }
  Workspace *W32 = (Workspace *)op32->sv_scal, *W64 = (Workspace *)op64->sv_scal;
  Scalars *S32 = &W32->S, *S64 = &W64->S;
  const bool v4 = use_v4<float>(n, x32, r32);
  const dim3 g(grid_vec(v4 ? n / 4 : n, nrhs), nrhs), g64(grid_vec(n, nrhs), nrhs);
  int *dflags = nullptr;
  if (cudaMalloc(&dflags, 16 * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return dg_record_error(DG_ERR_OOM); }
  std::vector<int> flags(nrhs, 1), converged(nrhs, 0), updates(nrhs, 0);
  std::vector<double> rr_ref(nrhs, 0.0), relres(nrhs, 1.0);
  Scalars h32, h64;
  cudaStream_t cs = s;
  bool own_stream = false;
  dg_status result = DG_ERR_NOT_CONVERGED;
  // FP64 residual of the current x: r64 = b - A64 x, its norm and ||b|| (into S64)
  auto true_residual = [&]() -> dg_status {
    dg_status e = dg_apply_internal(op64, x, ax64, nrhs, cs, false);
    if (e != DG_OK) return e;
    k_residual<double, false><<<g64, kThreads, 0, cs>>>(b, ax64, r64, n);
    k_dot<double, false><<<g64, kThreads, 0, cs>>>(r64, r64, W64->partial, n);
    k_reduce<<<nrhs, kThreads, 0, cs>>>(W64->partial, S64->rr, g64.x);
    SCK(cudaMemcpyAsync(&h64, S64, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
    SCK(cudaStreamSynchronize(cs));
    for (int i = 0; i < nrhs; ++i) {
      relres[i] = h64.bb[i] > 0 ? sqrt(h64.rr[i] / h64.bb[i]) : 0.0;
      converged[i] = relres[i] <= o.rtol;
    }
    return DG_OK;
  };
  // r32 = (float) r64, x32 = 0, and r.z, r.r of the new residual (the direction is kept)
  auto replace_residual = [&]() -> dg_status {
    k_to_float<<<grid_for((int64_t)nv), kThreads, 0, cs>>>(r64, r32, (int64_t)nv);
    SCK(cudaMemsetAsync(x32, 0, nv * sizeof(float), cs));
    if (z) {
      int nb = 0;
      SCK(launch_block_jacobi<float>(op32, op32->bj_tab.data(), (const float *)op32->d_bjinv, r32, z, nrhs,
                                     W32->partial, kMaxBlocks, &nb, cs));
      k_reduce<<<nrhs, kThreads, 0, cs>>>(W32->partial, S32->rz, nb);
      launch_dot<float>(v4, g, cs, r32, r32, W32->partial2, n);
      k_reduce<<<nrhs, kThreads, 0, cs>>>(W32->partial2, S32->rr, g.x);
    } else {
      k_refresh<float><<<g64, kThreads, 0, cs>>>(r32, dinv, W32->partial, W32->partial2, n);
      k_reduce<<<nrhs, kThreads, 0, cs>>>(W32->partial, S32->rz, g64.x);
      k_reduce<<<nrhs, kThreads, 0, cs>>>(W32->partial2, S32->rr, g64.x);
    }
    SCK(cudaGetLastError());
    return DG_OK;
  };
  do {
    if (o.use_graph && s == 0) {  // the legacy stream cannot be captured
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamSynchronize(0) != cudaSuccess) { result = dg_record_error(DG_ERR_CUDA); break; }
      own_stream = true;
    }
    k_zero_scalars<<<1, 128, 0, cs>>>(S64);
    k_dot<double, false><<<g64, kThreads, 0, cs>>>(b, b, W64->partial, n);
    k_reduce<<<nrhs, kThreads, 0, cs>>>(W64->partial, S64->bb, g64.x);
    if ((st = true_residual()) != DG_OK) { result = st; break; }
    // start: p = z = M^-1 r32 with the scalars of the FP32 recursion
    k_to_float<<<grid_for((int64_t)nv), kThreads, 0, cs>>>(r64, r32, (int64_t)nv);
    SCK(cudaMemsetAsync(x32, 0, nv * sizeof(float), cs));
    k_zero_scalars<<<1, 128, 0, cs>>>(S32);
    SCK(cudaMemcpyAsync(S32->bb, S64->bb, nrhs * sizeof(double), cudaMemcpyDeviceToDevice, cs));
    if ((st = start_directions<float>(op32, v4, g, r32, p, dinv, z, W32, nrhs, cs)) != DG_OK) { result = st; break; }
    // the FP32 recursion stops a right-hand side at half the target (then an update checks it)
    k_init_scalars<<<1, 32, 0, cs>>>(S32, nrhs, 0.5 * o.rtol);
    for (int i = 0; i < nrhs; ++i) flags[i] = !converged[i];
    SCK(cudaMemcpyAsync(dflags, flags.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, cs));
    k_set_active<<<1, 32, 0, cs>>>(S32, dflags, nrhs);
    SCK(cudaMemcpyAsync(&h32, S32, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
    SCK(cudaStreamSynchronize(cs));
    for (int i = 0; i < nrhs; ++i) rr_ref[i] = h32.rr[i];
    const int chunk = o.chunk > 0 ? o.chunk : 25;
    void *key = (void *)((uintptr_t)x32 ^ ((uintptr_t)r32 << 1) ^ ((uintptr_t)op32->kappa_vol << 2) ^
                         ((uintptr_t)dinv << 5) ^ ((uintptr_t)z << 7) ^ ((uintptr_t)nrhs << 48) ^
                         ((uintptr_t)chunk << 56) ^ (uintptr_t)0x5a5a);
    if (o.use_graph && (op32->sv_graph == nullptr || op32->sv_graph_key != key)) {
      drop_graph(op32);
      const bool prof = op32->prof;
      op32->prof = false;
      cudaGraph_t graph;
      SCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      dg_status est = enqueue<float>(v4, op32, x32, r32, p, Ap, dinv, z, W32, nrhs, chunk, cs);
      cudaError_t ce = cudaStreamEndCapture(cs, &graph);
      op32->prof = prof;
      if (est != DG_OK) { result = est; break; }
      if (ce != cudaSuccess) { result = dg_record_error(DG_ERR_CUDA); break; }
      cudaGraphExec_t exec;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) { result = dg_record_error(DG_ERR_CUDA); break; }
      op32->sv_graph = (void *)exec;
      op32->sv_graph_key = key;
    }
    bool all = true;
    for (int i = 0; i < nrhs; ++i) all = all && converged[i];
    int done = 0;
    while (!all && done < o.max_iters) {
      if (o.use_graph) {
        SCK(cudaGraphLaunch((cudaGraphExec_t)op32->sv_graph, cs));
      } else if ((st = enqueue<float>(v4, op32, x32, r32, p, Ap, dinv, z, W32, nrhs, chunk, cs)) != DG_OK) {
        result = st;
        break;
      }
      done += chunk;
      SCK(cudaMemcpyAsync(&h32, S32, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
      SCK(cudaStreamSynchronize(cs));
      bool update = done >= o.max_iters;
      for (int i = 0; i < nrhs; ++i)
        if (!converged[i] && (!h32.active[i] || h32.rr[i] <= delta * delta * rr_ref[i])) update = true;
      if (!update) continue;
      k_add_correction<<<grid_for((int64_t)nv), kThreads, 0, cs>>>(x, x32, (int64_t)nv);
      if ((st = true_residual()) != DG_OK) { result = st; break; }
      if ((st = replace_residual()) != DG_OK) { result = st; break; }
      all = true;
      for (int i = 0; i < nrhs; ++i) {
        flags[i] = !converged[i] && !h32.breakdown[i];
        if (!converged[i]) ++updates[i];
        all = all && converged[i];
      }
      SCK(cudaMemcpyAsync(dflags, flags.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, cs));
      k_set_active<<<1, 32, 0, cs>>>(S32, dflags, nrhs);
      SCK(cudaMemcpyAsync(&h32, S32, sizeof(Scalars), cudaMemcpyDeviceToHost, cs));
      SCK(cudaStreamSynchronize(cs));
      for (int i = 0; i < nrhs; ++i) rr_ref[i] = h32.rr[i];
    }
    if (st != DG_OK && result != DG_ERR_NOT_CONVERGED) break;
    result = all ? DG_OK : DG_ERR_NOT_CONVERGED;
    for (int i = 0; i < nrhs; ++i) {
      info[i].iters = h32.iters[i];
      info[i].outer = updates[i];
      info[i].converged = converged[i];
      info[i].breakdown = h32.breakdown[i];
      info[i].relres = relres[i];
    }
  } while (0);
  cudaFree(dflags);
  if (own_stream) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  return result;
}

}  // namespace

void dg_solver_release(dg_operator *op) {
  drop_graph(op);
  if (op->sv_vec) cudaFree(op->sv_vec);
  if (op->sv_aux) cudaFree(op->sv_aux);
  if (op->sv_scal) cudaFree(op->sv_scal);
  if (op->sv_dinv) cudaFree(op->sv_dinv);
  if (op->d_bjinv) cudaFree(op->d_bjinv);
  op->sv_vec = op->sv_aux = op->sv_scal = op->sv_dinv = op->d_bjinv = nullptr;
}

extern "C" {

dg_status dg_operator_diagonal(const dg_operator *op_c, void *diag, void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (!op || !diag || ((uintptr_t)diag & 15u)) return dg_record_error(DG_ERR_INVALID_ARG);
  if (op->problem != DG_SCALAR || op->aniso) return dg_record_error(DG_ERR_UNSUPPORTED);
  cudaStream_t s = (cudaStream_t)stream;
  if (op->precision == DG_FP64) return diagonal_by_colours<double>(op, (double *)diag, false, s);
  return diagonal_by_colours<float>(op, (float *)diag, false, s);
}

dg_status dg_operator_block_jacobi(const dg_operator *op_c, const void *r, void *z, int nrhs, void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (!op || !r || !z || r == z || nrhs < 1 || nrhs > op->max_rhs) return dg_record_error(DG_ERR_INVALID_ARG);
  if (((uintptr_t)r & 15u) || ((uintptr_t)z & 15u)) return dg_record_error(DG_ERR_INVALID_ARG);
  dg_status st = ensure_block_jacobi(op);
  if (st != DG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = op->precision == DG_FP64
                      ? launch_block_jacobi<double>(op, op->bj_tab.data(), (const double *)op->d_bjinv,
                                                    (const double *)r, (double *)z, nrhs, nullptr, 0, nullptr, s)
                      : launch_block_jacobi<float>(op, op->bj_tab.data(), (const float *)op->d_bjinv,
                                                   (const float *)r, (float *)z, nrhs, nullptr, 0, nullptr, s);
  return e == cudaSuccess ? DG_OK : dg_record_error(DG_ERR_CUDA);
}

dg_status dg_cg_solve(const dg_operator *op_c, const void *b, void *x, int nrhs, const dg_cg_options *opt,
                      dg_solve_info *info, void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (!op || !b || !x || !opt || !info || b == x) return dg_record_error(DG_ERR_INVALID_ARG);
  if (nrhs < 1 || nrhs > op->max_rhs || opt->max_iters < 1 || !(opt->rtol > 0)) return dg_record_error(DG_ERR_INVALID_ARG);
  if (opt->precond < DG_PRECOND_NONE || opt->precond > DG_PRECOND_BLOCK_JACOBI) return dg_record_error(DG_ERR_INVALID_ARG);
  if (((uintptr_t)b & 15u) || ((uintptr_t)x & 15u)) return dg_record_error(DG_ERR_INVALID_ARG);
  if (op->problem != DG_SCALAR || (op->aniso && opt->precond != DG_PRECOND_NONE)) return dg_record_error(DG_ERR_UNSUPPORTED);
  cudaStream_t s = (cudaStream_t)stream;
  dg_status st;
  if (op->precision == DG_FP64) st = cg_run<double>(op, (const double *)b, (double *)x, nrhs, *opt, false, true, info, s);
  else st = cg_run<float>(op, (const float *)b, (float *)x, nrhs, *opt, false, true, info, s);
  return st == DG_OK ? DG_OK : dg_record_error(st);
}

dg_status dg_refine_solve(const dg_operator *op64_c, const dg_operator *op32_c, const double *b, double *x, int nrhs,
                          double rtol, int max_outer, const dg_cg_options *inner, dg_solve_info *info, void *stream) {
  dg_operator *op64 = const_cast<dg_operator *>(op64_c), *op32 = const_cast<dg_operator *>(op32_c);
  if (!op64 || !op32 || !b || !x || !inner || !info || (const void *)b == (const void *)x) return dg_record_error(DG_ERR_INVALID_ARG);
  if (op64->precision != DG_FP64 || op32->precision != DG_FP32 || op64->ndofs != op32->ndofs) return dg_record_error(DG_ERR_INVALID_ARG);
  if (nrhs < 1 || nrhs > op64->max_rhs || nrhs > op32->max_rhs || max_outer < 1 || !(rtol > 0)) return dg_record_error(DG_ERR_INVALID_ARG);
  if (((uintptr_t)b & 15u) || ((uintptr_t)x & 15u)) return dg_record_error(DG_ERR_INVALID_ARG);
  if (op64->problem != DG_SCALAR || op32->problem != DG_SCALAR) return dg_record_error(DG_ERR_UNSUPPORTED);
  if ((op64->aniso || op32->aniso) && inner->precond != DG_PRECOND_NONE) return dg_record_error(DG_ERR_UNSUPPORTED);
  const int64_t n = op64->ndofs;
  const size_t nv = (size_t)nrhs * n;
  // FP64 residual and A x; FP32 right-hand side and correction of the inner solve
  const size_t need = nv * (2 * sizeof(double) + 2 * sizeof(float));
  if (op64->sv_aux_bytes < need) {
    if (op64->sv_aux) cudaFree(op64->sv_aux);
    op64->sv_aux = nullptr;
    op64->sv_aux_bytes = 0;
    if (cudaMalloc(&op64->sv_aux, need) != cudaSuccess) { cudaGetLastError(); return dg_record_error(DG_ERR_OOM); }
    op64->sv_aux_bytes = need;
  }
  if (!op64->sv_scal && cudaMalloc(&op64->sv_scal, sizeof(Workspace)) != cudaSuccess) {
    cudaGetLastError();
    return dg_record_error(DG_ERR_OOM);
  }
  double *r64 = (double *)op64->sv_aux, *ax64 = r64 + nv;
  float *r32 = (float *)(ax64 + nv), *d32 = r32 + nv;
  Workspace *W = (Workspace *)op64->sv_scal;
  Scalars *S = &W->S;
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 g(grid_vec(n, nrhs), nrhs);
  Scalars h;
  std::vector<int> inner_iters(nrhs, 0);
  dg_solve_info sub[16];
  int outer = 0;
  bool ok = false;
  for (;;) {
    // r = b - A x and its norm, in FP64
    dg_status st = dg_apply_internal(op64, x, ax64, nrhs, s, false);
    if (st != DG_OK) return dg_record_error(st);
    k_residual<double, false><<<g, kThreads, 0, s>>>(b, ax64, r64, n);
    k_zero_scalars<<<1, 128, 0, s>>>(S);
    k_dot<double, false><<<g, kThreads, 0, s>>>(b, b, W->partial, n);
    k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->bb, g.x);
    k_dot<double, false><<<g, kThreads, 0, s>>>(r64, r64, W->partial, n);
    k_reduce<<<nrhs, kThreads, 0, s>>>(W->partial, S->rr, g.x);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(&h, S, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    bool all = true;
    for (int i = 0; i < nrhs; ++i) {
      info[i].relres = h.bb[i] > 0 ? sqrt(h.rr[i] / h.bb[i]) : 0.0;
      info[i].converged = info[i].relres <= rtol;
      all = all && info[i].converged;
    }
    if (all) { ok = true; break; }
    if (outer >= max_outer) break;
    // inner FP32 CG on A d = r from d = 0; converged right-hand sides get r = 0
    for (int i = 0; i < nrhs; ++i) {
      if (info[i].converged) SCK(cudaMemsetAsync(r64 + (size_t)i * n, 0, n * sizeof(double), s));
    }
    k_to_float<<<grid_for((int64_t)nv), kThreads, 0, s>>>(r64, r32, (int64_t)nv);
    SCK(cudaMemsetAsync(d32, 0, nv * sizeof(float), s));
    st = cg_run<float>(op32, r32, d32, nrhs, *inner, true, false, sub, s);
    if (st != DG_OK && st != DG_ERR_NOT_CONVERGED) return dg_record_error(st);
    for (int i = 0; i < nrhs; ++i) inner_iters[i] += sub[i].iters;
    k_add_correction<<<grid_for((int64_t)nv), kThreads, 0, s>>>(x, d32, (int64_t)nv);
    SCK(cudaGetLastError());
    ++outer;
  }
  for (int i = 0; i < nrhs; ++i) {
    info[i].iters = inner_iters[i];
    info[i].outer = outer;
    info[i].breakdown = 0;
  }
  return ok ? DG_OK : dg_record_error(DG_ERR_NOT_CONVERGED);
}

dg_status dg_mixed_cg_solve(const dg_operator *op64_c, const dg_operator *op32_c, const double *b, double *x,
                            int nrhs, double delta, const dg_cg_options *opt, dg_solve_info *info, void *stream) {
  dg_operator *op64 = const_cast<dg_operator *>(op64_c), *op32 = const_cast<dg_operator *>(op32_c);
  if (!op64 || !op32 || !b || !x || !opt || !info || (const void *)b == (const void *)x) return dg_record_error(DG_ERR_INVALID_ARG);
  if (op64->precision != DG_FP64 || op32->precision != DG_FP32 || op64->ndofs != op32->ndofs) return dg_record_error(DG_ERR_INVALID_ARG);
  if (nrhs < 1 || nrhs > op64->max_rhs || nrhs > op32->max_rhs || !(opt->rtol > 0) || opt->max_iters < 1) return dg_record_error(DG_ERR_INVALID_ARG);
  if (!(delta > 0) || delta >= 1 || opt->precond < DG_PRECOND_NONE || opt->precond > DG_PRECOND_BLOCK_JACOBI) return dg_record_error(DG_ERR_INVALID_ARG);
  if (((uintptr_t)b & 15u) || ((uintptr_t)x & 15u)) return dg_record_error(DG_ERR_INVALID_ARG);
  if (op64->problem != DG_SCALAR || op32->problem != DG_SCALAR) return dg_record_error(DG_ERR_UNSUPPORTED);
  if ((op64->aniso || op32->aniso) && opt->precond != DG_PRECOND_NONE) return dg_record_error(DG_ERR_UNSUPPORTED);
  dg_status st = mixed_cg_run(op64, op32, b, x, nrhs, *opt, delta, info, (cudaStream_t)stream);
  return st == DG_OK ? DG_OK : dg_record_error(st);
}

}  // extern "C"
