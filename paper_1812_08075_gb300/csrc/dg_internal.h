// Internal declarations of libdg (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dg.h"

// Double-float number: the unevaluated sum hi + lo of two FP32 values with |lo| at most
// half an ulp of hi, about 48 significant bits and the FP32 exponent range. The kernel
// variant DG_VARIANT_DF64 runs the FP64 operator's three kernels in this arithmetic on the
// FP32 pipes (device arithmetic in dg_df64.cuh); its vectors stay FP64 in memory.
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

#ifdef __CUDACC__
// L2 prefetch of the bytes [p, p + n) that lie inside [lo, hi), rounded inwards to the
// 16-byte granularity of the bulk prefetch (one instruction, no registers held). Kernels
// use it for the inputs of the block that will run one wave after them.
__device__ __forceinline__ void dg_prefetch_l2(const void *lo, const void *hi, const void *p, size_t n) {
  uintptr_t a = (uintptr_t)p, e = a + n;
  const uintptr_t l = ((uintptr_t)lo + 15) & ~(uintptr_t)15, h = (uintptr_t)hi & ~(uintptr_t)15;
  a &= ~(uintptr_t)15;
  e = (e + 15) & ~(uintptr_t)15;
  if (a < l) a = l;
  if (e > h) e = h;
  if (e > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// v_i for a run-time i in {0, 1, 2}, by selects: indexing a local array with a run-time
// axis instead would place the array in local memory.
template <typename T>
__device__ __forceinline__ T dg_pick3(const T &v0, const T &v1, const T &v2, int i) {
  return i == 0 ? v0 : (i == 1 ? v1 : v2);
}

// Asynchronous copy of one 4-, 8- or 16-byte element global -> shared (cp.async): the
// thread issues it without waiting, and dg_cp_async_wait_all() waits for all of its own.
template <typename T>
__device__ __forceinline__ void dg_cp_async(T *dst, const T *src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"((int)sizeof(T))
               : "memory");
}
// 16 bytes at once (both addresses 16-byte aligned), bypassing L1
__device__ __forceinline__ void dg_cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void dg_cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
#endif

// Element type of the input and output vectors of kernels computing in T.
template <typename T>
struct IOType { using type = T; };
template <>
struct IOType<df64> { using type = double; };
template <typename T>
using io_t = typename IOType<T>::type;

#define DG_MAXP 6  // basis points per direction (degree <= 5)
#define DG_MAXM 7  // Gauss points per direction (k+1, or k+2 for over-integration)

// Reference-element tables in the operator's precision, uploaded once per operator.
// Internally the kernels work on values at the Gauss points (a collocated Lagrange
// basis on the Gauss nodes), which turns the derivative contractions into one
// m x m matrix per direction (see dg_tables.cpp).
template <typename T>
struct DevTables {
  T interp[DG_MAXM * DG_MAXP];  // [q][j] GLL basis j at Gauss point q
  T dcol[DG_MAXM * DG_MAXM];    // [q][r] d/dxi of Gauss-Lagrange basis r at Gauss point q
  T e0[DG_MAXM], e1[DG_MAXM];   // Gauss-Lagrange basis at xi = 0, 1
  T d0[DG_MAXM], d1[DG_MAXM];   // its derivative at xi = 0, 1
  T w[DG_MAXM];                 // Gauss weights on [0,1]
  T s[DG_MAXM];                 // Gauss nodes on [0,1]
  T gd0[DG_MAXP], gd1[DG_MAXP]; // derivative of the GLL basis at xi = 0, 1
  T interp_p[DG_MAXM * DG_MAXP];  // [q][l] pressure GLL basis (degree k-1) at Gauss point q
};

struct HostTables {
  int k, p, m;
  double gauss_s[DG_MAXM], gauss_w[DG_MAXM];
  double gll[DG_MAXP];
  double interp[DG_MAXM * DG_MAXP];
  double dcol[DG_MAXM * DG_MAXM];
  double e0[DG_MAXM], e1[DG_MAXM], d0[DG_MAXM], d1[DG_MAXM];
  double gd0[DG_MAXP], gd1[DG_MAXP];  // GLL basis derivative at xi = 0, 1
  // pressure space of the Stokes problem (degree k-1): GLL basis at the Gauss points
  int pp;
  double interp_p[DG_MAXM * DG_MAXP];
};

// Builds the tables for degree k (p = k+1 basis points) and m Gauss points; pressure
// degree k-1 tables when with_pressure. Returns 0 on success.
int dg_build_tables(int k, int m, bool with_pressure, HostTables *t);

// Geometry modes as seen by the kernels.
enum { GEO_AFFINE = 0, GEO_STORED = 1, GEO_RECOMPUTE = 2 };

// Everything the scalar kernels need, passed by value.
template <typename T>
struct ScalarArgs {
  int nx, ny, nz;
  int64_t ncell;
  int64_t nface;            // all faces of all three axes (interior and boundary)
  int64_t face_off[4];      // first face id of axis a; face_off[3] = nface
  const DevTables<T> *tab;
  // affine fast path (axis-parallel unit-cube lattice): per-axis constants
  T vol_g[3];               // detJ * (1/h_a)^2  (times the Gauss weight in-kernel)
  T vol_m;                  // c * detJ
  T vol;                    // detJ = 1 / (nx ny nz)
  T face_b[3];              // |F_a| / h_a : reference normal derivative weight
  T face_pw[3];             // gamma_a * |F_a|
  T face_area[3];           // |F_a| (face area element of the affine lattice)
  // stored geometry (GEO_STORED): gvol [ncell][7][m^3] = (G00,G01,G02,G11,G12,G22,mass)
  // with G = W detJ J^-1 J^-T and mass = c W detJ; gface [nface][7][m^2] =
  // (b-_0..2, b+_0..2, pw) with b = W J^-1 n_vec, pw = gamma W |n_vec|.
  const T *gvol;
  const T *gface;
  // recompute geometry (GEO_RECOMPUTE): vertex coordinates and per-face penalty
  const double *verts;
  const double *gamma_face; // [nface]
  double c;
  const io_t<T> *kappa_vol;   // [ncell][m^3] or NULL (FP64 for a double-float apply)
  const io_t<T> *kappa_face;  // [ncell][6][m^2] or NULL
  unsigned dmask;
  T sc, ss;                 // face flux / symmetry coefficients (forward: -1, theta)
};

// Launch shape of one kernel, filled instead of launching when a launcher gets a non-NULL
// query (used by the cost model): blocks launched, threads per block, resident blocks per
// SM (occupancy calculator) and, for persistent kernels, work items per launch.
struct LaunchInfo {
  int64_t blocks = 0;
  int threads = 0;
  int blocks_per_sm = 0;
  int64_t items = 0;
};

// Launchers (dg_scalar.cu). Return cudaError_t of the launch.
template <typename T>
cudaError_t launch_scalar_apply(int p, int m, int geo, bool kappa, const ScalarArgs<T> &a,
                                const io_t<T> *x, io_t<T> *y, T *rvol, T *traces, T *fres, int nrhs,
                                int64_t stride_dofs, int64_t stride_rvol, int64_t stride_tr,
                                int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev,
                                LaunchInfo *query = nullptr, int phases = 7, int64_t cell_begin = 0,
                                int64_t cell_count = -1, const HostTables *ht = nullptr);

// Adjoint of the scalar operator (dg_adjoint.cu, FP64): y = A^T r with a.sc/a.ss set for
// the transpose, and, when x is non-NULL, dkappa at every volume and face point for the
// forward form's theta (passed separately). Geometry is affine or recomputed from
// a.verts (geo = GEO_AFFINE or GEO_RECOMPUTE).
// nlmode 1 / 2 (with forward coefficients): the semilinear reaction's residual term
// beta (r^3, v) / Jacobian term 3 beta (x^2 r, v) added to the volume integral.
// T = double, or df64 (double-float arithmetic with FP64 vectors, kappa and dkappa).
// dk_acc: add dkappa to the arrays instead of overwriting them (sum over right-hand sides).
template <typename T>
cudaError_t launch_scalar_adjoint(int p, int geo, bool kappa, const ScalarArgs<T> &a, double theta,
                                  const io_t<T> *r, const io_t<T> *x, io_t<T> *y, io_t<T> *dk_vol,
                                  io_t<T> *dk_face, T *rvol, T *tr_r, T *tr_x, T *fres, int cpb, int fpb,
                                  cudaStream_t s, const cudaEvent_t *ev, int nlmode = 0, double beta = 0.0,
                                  bool dk_acc = false);

// Persistent single-pass apply for affine meshes (dg_fused.cu): one launch of one wave of
// blocks that loop over (right-hand side, row of cells) work items; each cell gathers its
// neighbours' face data from their coefficients, so no scratch memory is used.
template <typename T>
cudaError_t launch_fused_apply(int p, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                               int64_t stride_dofs, int tile, cudaStream_t s, const cudaEvent_t *ev, int *grid_out,
                               LaunchInfo *query = nullptr);

// One-thread-per-cell persistent apply for affine meshes, degree k <= 2 (dg_cellwise.cu):
// bricks of 8 x 4 x (cells / 32) cells per block, cells = 64, 128 or 256. dotp (FP32
// only): also the per-block partial sums of x . y per right-hand side, written to
// dotp[rhs * dot_stride + block] for block < *grid_out (dot_stride >= the grid).
template <typename T>
cudaError_t launch_cellwise_apply(int p, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                                  int64_t stride_dofs, int cells, cudaStream_t s, const cudaEvent_t *ev,
                                  int *grid_out, LaunchInfo *query = nullptr, double *dotp = nullptr,
                                  int dot_stride = 0);
size_t cellwise_smem_bytes(int p, int cells, int es);  // 0 if (p, cells) is not supported

// out[i] = in[i] as double-float (dg_scalar_df64.cu)
cudaError_t convert_to_df64(const double *in, df64 *out, int64_t n, cudaStream_t s);

// Cell-block Jacobi preconditioner by fast diagonalisation (dg_precond.cu): host tables
// (per axis and cell position, S and L; -1 if the operator is not affine scalar SIPG with
// kappa = 1, theta = -1 and k+1 points) and z = A_cc^-1 r with optional r.z partials.
struct dg_operator;
int block_jacobi_tables(const dg_operator *op, std::vector<double> &tab);
void block_jacobi_inverse_sums(int p, const std::vector<double> &tab, std::vector<double> &dinv);
template <typename T>
cudaError_t launch_block_jacobi(const dg_operator *op, const double *tab, const T *dinv, const T *r, T *z, int nrhs,
                                double *partial, int stride, int *blocks, cudaStream_t s);
// The same fused into preconditioned CG for FP32 operators with k <= 2 (block_jacobi_fusable):
//   BJ_UPDATE: r -= alpha Ap in place, z = A_cc^-1 r in registers, partials of r.z into prz
//     and of r.r into prr ([rhs * stride + block], *blocks blocks per right-hand side);
//   BJ_DIRECTION: z = A_cc^-1 r, x += alpha p, p = z + beta p (p only where active).
// alpha, beta, active: device arrays indexed by right-hand side.
enum { BJ_APPLY = 0, BJ_UPDATE = 1, BJ_DIRECTION = 2 };
bool block_jacobi_fusable(const dg_operator *op);
cudaError_t launch_block_jacobi_fused(const dg_operator *op, const double *tab, const float *dinv, int mode, float *r,
                                      const float *Ap, float *x, float *p, const double *alpha, const double *beta,
                                      const int *active, int nrhs, double *prz, double *prr, int stride, int *blocks,
                                      cudaStream_t s);

// Anisotropic degrees and quadrature (dg_aniso.cu): per-direction tables (host buffer of
// aniso_tab_bytes<T>() bytes; returns the trace words per cell) and the three-kernel apply
// with run-time extents; geo = GEO_AFFINE or GEO_RECOMPUTE (trilinear geometry from the
// vertices at every point); nq = m0 m1 m2 Gauss points per cell, npts = p0 p1 p2 DOFs.
template <typename T>
size_t aniso_tab_bytes();
template <typename T>
int aniso_tables(const HostTables ht[3], void *host_tab, int *trace_size);
template <typename T>
cudaError_t launch_aniso_apply(const ScalarArgs<T> &a, const void *dtab, int npts, int trace_size, const T *x, T *y,
                               T *rvol, T *traces, T *fres, int nrhs, int64_t sdof, int64_t srv, int64_t str,
                               int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev, int geo, bool kappa, int nq);
void aniso_work_model(const int kax[3], const int max[3], int geo, bool kappa, int64_t ncell, int64_t nface,
                      int64_t nbface, double flops[3], double bytes[3], int es);

// Stokes block operator (dg_stokes.cu), affine meshes: vector [u: ncell x 3 x P^3 | p: ncell x (P-1)^3];
// scratch rvol [ncell][4][M^3], traces and fres [ncell][42][M^2] per right-hand side.
template <typename T>
cudaError_t launch_stokes_apply(int p, const ScalarArgs<T> &a, T mu, const io_t<T> *x, io_t<T> *y, T *rvol, T *traces,
                                T *fres, int nrhs, int64_t stride_dofs, int64_t stride_rvol, int64_t stride_tr,
                                int cpb, int fpb, cudaStream_t s, const cudaEvent_t *ev);

// Data terms of the residual (dg_rhs.cu): F from f at the volume points and g at the
// boundary face points; geo = GEO_AFFINE or GEO_RECOMPUTE.
template <typename T>
cudaError_t launch_rhs(int p, int geo, bool kappa, const ScalarArgs<T> &a, T theta, const T *f, const T *g, T *F,
                       T *rvol, T *fres, int cpb, int fpb, cudaStream_t s);

// Geometry precompute (dg_geometry.cu).
template <typename T>
cudaError_t launch_geometry(int m, const ScalarArgs<T> &a, const double *verts, double c,
                            const double *gamma_face, const double *gauss_s, const double *gauss_w,
                            T *gvol, T *gface, cudaStream_t s);
cudaError_t launch_penalty(int m, int k, int pen_mode, double alpha, int nx, int ny, int nz,
                           int64_t nface, const int64_t *face_off, const double *verts,
                           const double *gauss_s, const double *gauss_w, double *gamma_face,
                           double *cell_vol, cudaStream_t s);

// Work model of the fused single-pass variant, per right-hand side (all in flops[0]).
void fused_work_model(int p, int64_t ncell, int64_t nbface, double flops[3], double bytes[3], int elem_size);
void cellwise_work_model(int p, int nx, int ny, int nz, int brick, int64_t nbface, double flops[3], double bytes[3],
                         int elem_size);

// Work model of the Stokes apply (op counts of the kernels), per right-hand side.
void stokes_work_model(int p, int64_t ncell, int64_t nface, int64_t nbface, double flops[3], double bytes[3],
                       int elem_size);

// Work model of the scalar apply (exact op counts of the kernels), per right-hand side.
void scalar_work_model(int p, int m, int geo, bool kappa, int64_t ncell, int64_t nface,
                       int64_t nbface, double flops[3], double bytes[3], int elem_size);


struct dg_mesh {
  int nx, ny, nz;
  bool affine;
  std::vector<double> verts;
};

struct dg_operator {
  int nx, ny, nz;
  int k, p, m;
  int problem, precision, max_rhs, geo;
  unsigned dmask;
  double c, mu, theta;
  dg_penalty pen;
  int64_t ncell, nface, nbface, ndofs;
  int64_t face_off[4];
  HostTables ht;
  void *d_tab = nullptr;
  double *d_verts = nullptr;
  double *d_gamma = nullptr;
  double *d_cellvol = nullptr;
  void *d_gvol = nullptr, *d_gface = nullptr;
  void *d_rvol = nullptr, *d_tr = nullptr, *d_fres = nullptr;
  void *d_xh = nullptr, *d_yh = nullptr;  // staging for dg_apply_host
  cudaStream_t hs_copy = nullptr;         // dg_apply_host: copy stream and its events (first use)
  std::vector<cudaEvent_t> hs_ev;
  void *d_tr2 = nullptr;                  // traces of x in the adjoint (allocated on first use)
  const void *kappa_vol = nullptr, *kappa_face = nullptr;
  int cpb = 1, fpb = 1;
  int variant = DG_VARIANT_THREE_KERNEL;  // resolved (never AUTO)
  int tile = 8;                          // cells per row tile of the fused kernel
  int brick = 128;                       // cells per brick of the cellwise kernel
  int fused_grid = 0;
  double gamma_axis[3];
  // per-kernel event timing (dg_operator_profile)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;  // 4 events per recorded apply
  size_t prof_used = 0;              // applies recorded since the last read
  // solver workspace (dg_solve.cu), allocated on the first solve and kept
  void *sv_vec = nullptr;   // vectors in the operator's precision
  size_t sv_vec_bytes = 0;
  void *sv_aux = nullptr;   // FP64 vectors of the refinement loop
  size_t sv_aux_bytes = 0;
  void *sv_scal = nullptr;  // per right-hand-side scalars
  void *sv_dinv = nullptr;  // inverse diagonal of A (Jacobi preconditioner), operator precision
  std::vector<double> bj_tab;  // block-Jacobi tables (empty until first use)
  // anisotropic degrees (dg_operator_create_aniso): per-direction tables on the device,
  // points per cell and trace words per cell; the isotropic fields describe k_max
  int aniso = 0;
  int kax[3] = {0, 0, 0};
  int max_q[3] = {0, 0, 0};  // Gauss points per direction
  int an_nq = 0;             // m0 m1 m2
  void *d_antab = nullptr;
  int an_npts = 0, an_ts = 0;
  void *d_bjinv = nullptr;     // their inverse eigenvalue sums on the device, operator precision
  // DG_VARIANT_DF64: tables and stored geometry as double-float (built on first use)
  void *d_tab_df = nullptr, *d_gvol_df = nullptr, *d_gface_df = nullptr;
  void *sv_graph = nullptr; // cached CUDA graph of a chunk of CG iterations (cudaGraphExec_t)
  void *sv_graph_key = nullptr;
};


// Multiprocessors of the current device (1 if the query fails); sizes grids and waves.
int dg_device_sms();

// Shared by the API and the solver (dg_api.cu).
dg_status dg_record_error(dg_status s);
dg_status dg_apply_internal(const dg_operator *op, const void *x, void *y, int nrhs, cudaStream_t s, bool transpose);
// y = A x with the per-block partial sums of x . y per right-hand side in
// dot_partial[rhs * dot_stride + block], block < *nblocks, where the operator's kernel
// computes them in the same pass (the FP32 cellwise variant). Otherwise launches nothing
// and returns DG_ERR_UNSUPPORTED without recording an error.
dg_status dg_apply_dot_internal(const dg_operator *op, const void *x, void *y, int nrhs, cudaStream_t s,
                                double *dot_partial, int dot_stride, int *nblocks);
void dg_solver_release(dg_operator *op);
