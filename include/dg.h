/*
 * dg.h - C ABI of libdg, a single-GPU (GB300, sm_103a) matrix-free application of the
 * symmetric interior-penalty Discontinuous Galerkin (SIPG) operator of
 *   Kempf, Hess, Muething, Bastian, "Automatic Code Generation for High-Performance
 *   Discontinuous Galerkin Methods on Modern Architectures", arXiv 1812.08075,
 * on structured hexahedral meshes with the tensor-product Q_k basis, evaluated by sum
 * factorisation (Sec. 2.2, Eq. lowcomplex, Algorithm 1).
 *
 * Conventions shared by every entry point
 *   - All compute entry points are asynchronous on the caller's CUDA stream (passed as
 *     `void* stream`, a cudaStream_t; NULL = the legacy default stream). Argument errors
 *     are reported immediately and enqueue nothing. Asynchronous CUDA errors surface on
 *     the next call or through dg_get_last_error(). No C++ exception crosses the ABI.
 *   - Device vectors are caller-owned, contiguous, 16-byte aligned and of the operator's
 *     precision (double for DG_FP64, float for DG_FP32). Outputs must not alias inputs.
 *   - Scalar DOF vector layout: cell-major [ncell][(k+1)^3], cells lexicographic
 *     c = cx + nx*(cy + ny*cz), cell DOFs j0 + p*(j1 + p*j2) (x fastest), on the
 *     Lagrange basis of the k+1 Gauss-Lobatto-Legendre points of [0,1] (the paper leaves
 *     the basis open, Sec. 2.1). Stokes: [u: ncell x 3 x (k+1)^3 | p: ncell x k^3].
 *     nrhs vectors are stored back to back, [nrhs][ndofs].
 *   - Calls on one operator must be ordered on one stream at a time: the operator owns
 *     scratch buffers that each apply reuses.
 *   - Every object is owned by the library from *_create until *_destroy.
 */
#ifndef DG_H
#define DG_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_INVALID_ARG = 1,   /* null pointer, bad size, misaligned or aliased buffer */
  DG_ERR_UNSUPPORTED = 2,   /* valid request outside what is built (e.g. degree > 5) */
  DG_ERR_OOM = 3,           /* device or host allocation failed */
  DG_ERR_CUDA = 4,          /* a CUDA runtime call failed (sticky; see dg_get_last_error) */
  DG_ERR_NOT_CONVERGED = 5, /* an iterative solve hit its iteration limit */
  DG_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up */
} dg_status;

typedef struct dg_mesh dg_mesh;
typedef struct dg_operator dg_operator;

enum { DG_PEN_CONFIG = 0, DG_PEN_PAPER = 1 };
enum { DG_SCALAR = 0, DG_STOKES = 1 };
enum { DG_FP64 = 0, DG_FP32 = 1 };
enum { DG_GEOM_AUTO = 0, DG_GEOM_STORED = 1, DG_GEOM_RECOMPUTE = 2 };
enum { DG_VARIANT_AUTO = 0, DG_VARIANT_THREE_KERNEL = 1, DG_VARIANT_FUSED = 2, DG_VARIANT_CELLWISE = 3, DG_VARIANT_DF64 = 4 };
enum { DG_PRECOND_NONE = 0, DG_PRECOND_JACOBI = 1, DG_PRECOND_BLOCK_JACOBI = 2 };
enum { DG_SEMILINEAR_RESIDUAL = 1, DG_SEMILINEAR_JACOBIAN = 2 };

/* Interior-penalty factor gamma_F (Sec. 5.2).
 *   DG_PEN_CONFIG: gamma_F = alpha * k * (k+1) / h_a with h_a = 1/n_a the nominal cell
 *                  size across the face (n_a cells along the face normal's axis);
 *   DG_PEN_PAPER:  gamma_F = alpha * k * (k+d-1) * |F| / min(|T+|, |T-|) (boundary:
 *                  |F|/|T|), measures by the operator's Gauss rule; the paper uses
 *                  alpha = 3. */
typedef struct {
  int32_t mode;
  int32_t reserved;
  double alpha;
} dg_penalty;

/* Coefficients and options of one operator.
 *   problem        DG_SCALAR: -div(kappa grad u) + c u (Eq. diffreac_weak);
 *                  DG_STOKES: -mu Lap u + grad p, div u (Eq. stokes_weak).
 *   precision      DG_FP64 or DG_FP32 (storage and arithmetic of the apply).
 *   dirichlet_mask bit lf set: domain face lf (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z) carries
 *                  the Dirichlet face terms; other boundary faces carry none.
 *   max_rhs        1..16, the largest nrhs any apply on this operator will use.
 *   geometry       DG_GEOM_AUTO / STORED (per-quadrature-point geometry precomputed once)
 *                  / RECOMPUTE (from vertex coordinates inside the kernels; scalar problem
 *                  with k+1 points, FP64 or FP32); ignored on affine meshes.
 *   c              reaction coefficient (scalar), mu viscosity (Stokes),
 *   theta          -1 symmetric (SIPG, the paper's choice), 0 incomplete, +1 non-symmetric. */
typedef struct {
  int32_t problem;
  int32_t precision;
  int32_t dirichlet_mask;
  int32_t max_rhs;
  int32_t geometry;
  int32_t reserved;
  double c;
  double mu;
  double theta;
} dg_coefficients;

/* Per-apply work model of an operator (exact counts of what the kernels execute).
 * flops[i] and bytes[i] are per right-hand side for kernel i of the apply
 * (0: cell/volume kernel, 1: face kernel, 2: back-projection kernel); bytes are the
 * algorithmic global-memory bytes (each input read once, each output written once). */
typedef struct {
  int64_t ndofs;
  int64_t ncell;
  int64_t nface;
  double flops[3];
  double bytes[3];
  double dofs_bytes;      /* x read + y written, per right-hand side */
  int32_t cells_per_block;
  int32_t faces_per_block;
  int32_t threads_cell;
  int32_t threads_face;
  int32_t geometry;       /* DG_GEOM_* in effect (0 = affine fast path) */
  int32_t variant;        /* DG_VARIANT_THREE_KERNEL, _FUSED, _CELLWISE or _DF64 */
  int32_t persistent_grid;/* blocks of the last fused (persistent) launch, 0 if none yet */
  int32_t reserved;
} dg_stats;

/* Human-readable name of a status code (static string). */
const char *dg_status_string(dg_status s);

/* Last error recorded by any call on this thread (DG_OK if none); clears it. */
dg_status dg_get_last_error(void);

/* Structured nx x ny x nz hexahedral mesh of cuboid cells (Sec. 2.1).
 * vertices: host array [(nx+1)(ny+1)(nz+1)][3] (v = i + (nx+1)(j + (ny+1) l)), copied;
 *           NULL = uniform unit cube (affine, axis-parallel cells, the fast path).
 * Each cell T is the image of [0,1]^3 under the trilinear map through its 8 vertices.
 * Errors: DG_ERR_INVALID_ARG (n < 1, out NULL), DG_ERR_OOM. */
dg_status dg_mesh_create(int nx, int ny, int nz, const double *vertices, dg_mesh **out);
dg_status dg_mesh_destroy(dg_mesh *mesh);

/* Operator y = A x of Eq. (diffreac_weak) or Eq. (stokes_weak) without the data terms
 * (the Jacobian action for a linear problem, Sec. 2.1), degree k (1..5 scalar, 2..5
 * Stokes), quad_points_1d Gauss-Legendre points per direction (0 = k+1; k+2 over-
 * integrates the scalar operator on the three-kernel path; the fused variant, Stokes,
 * the adjoint and dg_rhs need k+1). Uploads reference tables, precomputes geometry if stored, allocates scratch
 * for max_rhs right-hand sides. Synchronous. Errors: DG_ERR_INVALID_ARG,
 * DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_operator_create(const dg_mesh *mesh, int degree, int quad_points_1d,
                             const dg_penalty *penalty, const dg_coefficients *coef,
                             dg_operator **out);
dg_status dg_operator_destroy(dg_operator *op);

/* Scalar operator with anisotropic degrees and quadrature (Sec. 2.1: a degree k_a and a
 * Gauss rule of m_a points per direction; Sec. 4 raises m on purpose): degrees[a] = k_a in
 * 1..5, quad_points[a] = m_a with k_a + 1 <= m_a <= 7 (NULL or 0 entries: m_a = k_a + 1);
 * k_a + 1 GLL basis points per direction, cell DOFs j0 + p0 (j1 + p1 j2). The face penalty
 * takes the degree along the face normal (DG_PEN_CONFIG: alpha k_a (k_a + 1) / h_a;
 * DG_PEN_PAPER: alpha k_a (k_a + 2) / h_a, affine meshes only). Affine meshes and trilinear
 * meshes (geometry recomputed from the vertex coordinates at every point inside the
 * kernels; nothing stored), the scalar problem, FP64 or FP32. kappa (dg_operator_set_kappa)
 * then uses the per-direction layouts kappa_vol [ncell][m0 m1 m2] (q0 + m0 (q1 + m1 q2))
 * and kappa_face [ncell][sum over lf = 0..5 of m_t1 m_t2] (faces in order, points qs + m_t1 qt
 * over the tangential axes t1 < t2). The apply runs the three-kernel structure with run-time
 * extents. dg_apply, dg_apply_host, dg_operator_stats and unpreconditioned dg_cg_solve /
 * dg_refine_solve accept it; the adjoint, dg_rhs, dg_apply_semilinear, the preconditioners,
 * variants and the tuners return DG_ERR_UNSUPPORTED. Errors: DG_ERR_INVALID_ARG (k_a or m_a
 * out of range), DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_operator_create_aniso(const dg_mesh *mesh, const int32_t degrees[3],
                                   const int32_t quad_points[3], const dg_penalty *penalty,
                                   const dg_coefficients *coef, dg_operator **out);

/* Number of DOFs of one vector of this operator. */
dg_status dg_operator_ndofs(const dg_operator *op, int64_t *n);

/* Work model and launch configuration currently in effect (host only). */
dg_status dg_operator_stats(const dg_operator *op, dg_stats *out);

/* Kernel variant and blocking of later applies (the search space of the tuner).
 *   DG_VARIANT_THREE_KERNEL: cell kernel (volume terms and face traces), face kernel,
 *     back-projection kernel, with scratch for traces and residuals; any geometry.
 *   DG_VARIANT_FUSED: one persistent launch (one wave of blocks looping over
 *     (right-hand side, row of cells) items) in which each cell evaluates its faces from
 *     its own side with the neighbour's trace gathered from its coefficients; affine
 *     scalar operators without kappa only; no scratch.
 *   DG_VARIANT_CELLWISE: one persistent launch with one thread per cell: a block owns a
 *     brick of 8 x 4 x (cells_per_block / 32) cells (cells_per_block = 64, 128 or 256),
 *     each cell's sum factorisation runs in registers and the cells of a brick exchange
 *     face traces through shared memory; neighbours across the brick boundary are
 *     evaluated from their coefficients. Same operators as the fused variant, degree
 *     k <= 2; no scratch.
 *   DG_VARIANT_DF64: the three kernels of an FP64 operator computing in double-float
 *     arithmetic (each value an unevaluated sum of two FP32 numbers, about 48 significant
 *     bits, built from error-free FP32 transformations) on the FP32 pipes, which run at
 *     64 times the FP64 rate of this GPU. Vectors stay FP64 in memory and are converted
 *     on load and store; tables and stored geometry get double-float copies on the first
 *     use of the variant. FP64 Stokes operators and FP64 scalar operators (any
 *     geometry and kappa; with recomputed geometry, and for dg_apply_adjoint and
 *     dg_apply_semilinear, the adjoint kernels run in double-float too); the
 *     result agrees with the FP64 variant to a few 1e-14 relative. Never chosen by
 *     DG_VARIANT_AUTO; dg_operator_autotune keeps it and tunes its blockings.
 *   DG_VARIANT_AUTO: cellwise for FP32 affine scalar operators of degree k <= 2, fused
 *     for other FP32 affine scalar operators, three-kernel otherwise.
 * cells_per_block (cells per block, cells per row tile of the fused kernel, or cells per
 * brick of the cellwise kernel) and faces_per_block: 0 keeps the default. Errors:
 * DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED (a variant on an operator it does not cover,
 * blocking over the shared-memory limit or not a brick size). */
dg_status dg_operator_set_variant(dg_operator *op, int variant, int cells_per_block, int faces_per_block);

/* Result of dg_operator_autotune. ms_* are CUDA-event times of one apply of nrhs
 * right-hand sides; candidates counts the configurations timed. */
typedef struct {
  int32_t variant;
  int32_t cells_per_block;
  int32_t faces_per_block;
  int32_t candidates;
  double ms_best;
  double ms_default;
} dg_tune_result;

/* Measured tuning of the variant and blocking (Sec. 4's autotuning cost function, with
 * its divide-and-conquer search adapted): the cell-side blocking (cell and
 * back-projection kernels) and the face blocking are independent subproblems, each timed
 * per kernel with CUDA events over a few applies and minimised separately, then combined
 * and compared with the fused variant where it applies; the fastest is kept (as with
 * dg_operator_set_variant). Allocates and frees two scratch vectors of nrhs x ndofs;
 * synchronises the stream. Errors: DG_ERR_INVALID_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_operator_autotune(dg_operator *op, int nrhs, void *stream, dg_tune_result *out);

/* Launch cost model (Sec. 4's heuristic cost function cost = flops x ilp x loads, with
 * ilp = 1 + c0 log2(s), loads = 1 + c1 log2(p), c0 = 0.5, c1 = 0.25, carried to the GPU):
 * the predicted milliseconds of one apply of nrhs right-hand sides of the scalar operator
 * in the given configuration (variant DG_VARIANT_THREE_KERNEL with cells_per_block and
 * faces_per_block, or DG_VARIANT_FUSED / DG_VARIANT_CELLWISE with cells_per_block the
 * row tile / brick). Per kernel: the roofline time max(flops / peak of the precision,
 * bytes / HBM bandwidth) from the operator's exact work model, times 1 + c0 log2(16 / w)
 * for w < 16 resident warps per SM (the occupancy calculator's figure for the kernel at
 * that blocking), times the loads term with p = k+1, times the tail of the last partly
 * empty wave, plus 50 ns per block (per work item of a persistent kernel) and SM for what
 * each block loads before its first useful operation. It ranks the blockings of one
 * variant; it does not capture the latency-bound efficiency of the persistent FP32
 * variants, so choices between variants are measured. Launches nothing. Errors: DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED (Stokes,
 * recomputed geometry, a variant or blocking the operator does not cover), DG_ERR_CUDA. */
dg_status dg_operator_predict(const dg_operator *op, int nrhs, int variant, int cells_per_block,
                              int faces_per_block, double *ms);

/* Mean CUDA-event milliseconds of one apply of nrhs right-hand sides in the given
 * configuration (arguments as dg_operator_predict), on scratch vectors the call allocates
 * and frees; the operator's own configuration is unchanged. Synchronises the stream.
 * Errors: DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_operator_time(const dg_operator *op, int nrhs, int variant, int cells_per_block,
                           int faces_per_block, void *stream, double *ms);

/* Tuner with the cost model as prior: ranks the candidate blockings of each variant the
 * scalar operator supports by dg_operator_predict, times the first `measure` of each
 * variant and keeps the fastest timed configuration.
 * out->candidates = configurations timed, ms_best = the kept one's time, ms_default = the
 * model's prediction for its own first choice. Errors as dg_operator_autotune, and
 * DG_ERR_UNSUPPORTED for Stokes and recomputed geometry. */
dg_status dg_operator_autotune_prior(dg_operator *op, int nrhs, int measure, void *stream,
                                     dg_tune_result *out);

/* Per-quadrature-point diffusion coefficient kappa (scalar problem; anisotropic operators:
 * the per-direction layouts of dg_operator_create_aniso): device arrays of
 * the operator's precision, kappa_vol [ncell][m^3] (points q0 + m(q1 + m q2)) and
 * kappa_face [ncell][6][m^2] (each cell's own side of faces -x,+x,-y,+y,-z,+z, points
 * qs + m*qt over the two tangential axes in increasing order). NULL = 1. The arrays
 * are read at every apply (not copied) and must stay valid until the last apply that
 * uses them. The penalty does not involve kappa (Sec. 5.2). */
dg_status dg_operator_set_kappa(dg_operator *op, const void *kappa_vol, const void *kappa_face);

/* y = A x for nrhs (1..max_rhs) vectors (Sec. 2.1 Jacobian action; Algorithm 1 per
 * cell, facet sum factorisation per face). x, y: device [nrhs][ndofs]. y is
 * overwritten. Errors: DG_ERR_INVALID_ARG, DG_ERR_CUDA. */
dg_status dg_apply(const dg_operator *op, const void *x, void *y, int nrhs, void *stream);

/* Same operator applied through host buffers: copies x (host [nrhs][ndofs]) to the
 * device, applies, copies y back and synchronises the stream. Page-locked host memory
 * gives the full link bandwidth; pageable memory also works. For the three-kernel scalar
 * apply (FP64, FP32 or double-float; affine or stored geometry) the call pipelines over
 * eight chunks of cells: each chunk's x is copied ahead of its cell kernel and its y
 * behind its back-projection kernel, on an internal copy stream ordered by events, so
 * the copies overlap the kernels. The result is the same as dg_apply's. */
dg_status dg_apply_host(const dg_operator *op, const void *x_host, void *y_host, int nrhs,
                        void *stream);

/* Semilinear reaction: the operator of Eq. (diffreac_weak) plus a cubic reaction
 * beta (u^3, v) (the paper discusses the Jacobian action of nonlinear problems in Sec. 3
 * without fixing one; this is the reading chosen here). One vector, FP64 scalar operators
 * with k+1 points; geometry affine or recomputed in the kernels (trilinear meshes); kappa
 * honoured.
 *   DG_SEMILINEAR_RESIDUAL: y = A w + beta (w^3, v), the residual operator at w (u0 unused);
 *   DG_SEMILINEAR_JACOBIAN: y = A w + 3 beta (u0^2 w, v), its Jacobian action at the
 *     linearisation point u0 on the direction w: u0 and w are evaluated at the Gauss
 *     points in the same kernel (Sec. 3's two-input fusion).
 * w, u0, y: device [ndofs] FP64, 16-byte aligned, y distinct from both. Errors:
 * DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED (Stokes, FP32, over-integration), DG_ERR_CUDA. */
dg_status dg_apply_semilinear(const dg_operator *op, int mode, double beta, const void *u0,
                              const void *w, void *y, void *stream);

/* Data terms of Eq. (diffreac_weak) moved to the right-hand side (scalar problem):
 *   F(v) = (f, v) + theta (g, n.kappa grad v)_{Gamma_D} + gamma_F (g, v)_{Gamma_D},
 * so that the residual of Sec. 2.1 is r(u) = A u - F and the discrete problem A u = F.
 * f_vol: f at the volume Gauss points, device [ncell][m^3] (points q0 + m(q1 + m q2)),
 * NULL = 0; g_face: Dirichlet data at each cell's face Gauss points, device
 * [ncell][6][m^2] (layout of kappa_face), read only on Dirichlet boundary faces, NULL = 0.
 * kappa as set by dg_operator_set_kappa. F: device [ndofs], overwritten. Uses the
 * operator's scratch (ordered with applies on one stream). Trilinear geometry is
 * recomputed from the vertices. Errors: DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED (Stokes),
 * DG_ERR_CUDA. */
dg_status dg_rhs(const dg_operator *op, const void *f_vol, const void *g_face, void *F, void *stream);

/* Adjoint of the scalar operator for the loss L = 0.5 sum_s ||A(kappa) x_s - b_s||^2 over
 * nrhs right-hand sides (Sec. 2.1: the transposed Jacobian action of the linear problem):
 *   y_s = A^T r_s for s = 0..nrhs-1 (the transposed apply, r_s = A x_s - b_s supplied by the
 *   caller), and, when x and the output arrays are non-NULL,
 *   dkappa_vol[c][q] = sum_s r_s^T dA/dkappa_vol[c][q] x_s and dkappa_face[c][lf][q] likewise
 *   (layouts as dg_operator_set_kappa; one array shared by all right-hand sides, holding
 *   the gradient of the summed loss).
 * r, x, y: device [nrhs][ndofs], nrhs in 1..max_rhs; y distinct from r and x.
 * Geometry is recomputed from the vertex coordinates inside the kernels (nothing
 * stored is required). Stokes and FP32 operators give y = A^T r only (their forward
 * kernels with the flux and symmetry coefficients exchanged; the Stokes coupling is its
 * own transpose), and require dkappa NULL. Errors: DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED
 * (dkappa on Stokes or FP32, anisotropic degrees, over-integration), DG_ERR_OOM (the
 * first call with dkappa allocates a second trace buffer), DG_ERR_CUDA. */
dg_status dg_apply_adjoint(const dg_operator *op, const void *r, const void *x, void *y,
                           void *dkappa_vol, void *dkappa_face, int nrhs, void *stream);

/* Options of the conjugate-gradient solves (the paper has no solver; these are the
 * solves the matrix-free apply serves).
 *   rtol       stop a right-hand side when ||b - A x||_2 <= rtol ||b||_2
 *   max_iters  iteration limit (rounded up to a multiple of chunk)
 *   chunk      iterations enqueued between host convergence checks (0 = 25)
 *   use_graph  1: capture one chunk into a CUDA graph on the first call and replay it
 *   precond    DG_PRECOND_NONE; DG_PRECOND_JACOBI (point Jacobi with diag(A) from
 *              dg_operator_diagonal, computed on first use and kept by the operator
 *              until its kappa changes); or DG_PRECOND_BLOCK_JACOBI (the cell blocks of
 *              A inverted by dg_operator_block_jacobi; operators it covers only) */
typedef struct {
  double rtol;
  int32_t max_iters;
  int32_t chunk;
  int32_t use_graph;
  int32_t precond;
} dg_cg_options;

/* diag(A) of the scalar operator (device [ndofs], operator precision): A is applied to
 * unit vectors of one cell colour (the 8 parity classes of the cell coordinates, which
 * share no face) and one local DOF at a time, 8 (k+1)^3 applies in all. Allocates and
 * frees two vectors; synchronises the stream. The paper has no preconditioner; this is
 * the point-Jacobi preconditioner of the solves below. Errors: DG_ERR_INVALID_ARG,
 * DG_ERR_UNSUPPORTED (Stokes), DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_operator_diagonal(const dg_operator *op, void *diag, void *stream);

/* Cell-block Jacobi preconditioner: z_c = A_cc^-1 r_c for every cell c, where A_cc is the
 * diagonal block of cell c (the volume terms of Eq. diffreac_weak and the cell's own side
 * of its six faces). On affine cells with kappa = 1 that block is a Kronecker sum of 1D
 * matrices (Sec. 2.2's tensor structure), so it is inverted exactly by fast
 * diagonalisation: generalized eigenvectors of the 1D stiffness-plus-face matrix and the
 * 1D mass matrix per axis and cell position (computed on the host in FP64 on first use),
 * then three transposed sweeps, a pointwise division and three sweeps per cell (the
 * paper has no preconditioner). r, z: device [nrhs][ndofs], operator precision, distinct.
 * Errors: DG_ERR_INVALID_ARG; DG_ERR_UNSUPPORTED unless the operator is scalar, affine,
 * without kappa, theta = -1 and k+1 points per direction; DG_ERR_CUDA. */
dg_status dg_operator_block_jacobi(const dg_operator *op, const void *r, void *z, int nrhs, void *stream);

/* Per right-hand-side result of a solve. iters: CG iterations (summed over the inner
 * solves of a refinement); outer: refinement steps; relres: final ||b - A x|| / ||b||
 * (for refinement recomputed in FP64); breakdown: CG met p.Ap <= 0. */
typedef struct {
  int32_t iters;
  int32_t outer;
  int32_t converged;
  int32_t breakdown;
  double relres;
} dg_solve_info;

/* Batched (optionally point- or block-Jacobi-preconditioned) conjugate gradients on A x = b (scalar operator, SPD for
 * theta = -1 with penalty large enough): nrhs (1..max_rhs) independent solves advanced
 * together, vectors in the operator's precision, dot products accumulated in FP64,
 * per right-hand-side scalars kept on the device. x (device [nrhs][ndofs]) holds the
 * initial guess and receives the solution; b and x must not alias. info has nrhs
 * entries. When the recursively updated residual meets rtol, the true residual b - A x is
 * recomputed and the solve continues from it (at most 3 times) where it does not. Workspace (4 vectors x max_rhs) is allocated on the first call and kept by
 * the operator. Synchronises the stream before returning. Errors: DG_ERR_INVALID_ARG,
 * DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NOT_CONVERGED (info filled). */
dg_status dg_cg_solve(const dg_operator *op, const void *b, void *x, int nrhs,
                      const dg_cg_options *opt, dg_solve_info *info, void *stream);

/* Mixed-precision iterative refinement: repeat r = b - A64 x (FP64), stop when
 * ||r|| <= rtol ||b|| for every right-hand side, else solve A32 d = (float) r by the
 * batched FP32 CG above to inner->rtol and update x += d in FP64. op64 (DG_FP64) and
 * op32 (DG_FP32) must discretise the same operator. b, x: FP64 device [nrhs][ndofs];
 * x holds the initial guess. Errors as dg_cg_solve. */
dg_status dg_refine_solve(const dg_operator *op64, const dg_operator *op32, const double *b,
                          double *x, int nrhs, double rtol, int max_outer,
                          const dg_cg_options *inner, dg_solve_info *info, void *stream);

/* Mixed-precision CG with reliable updates (residual replacement): FP32 CG iterations with
 * op32 (batched, chunks captured in a CUDA graph as in dg_cg_solve, FP64 inner products,
 * optional preconditioner) that continue across updates. An update adds the FP32 correction
 * to the FP64 solution x, recomputes the residual b - A x in FP64 with op64, and replaces
 * the FP32 residual by it while keeping the search direction; it runs at the end of a chunk
 * when a right-hand side's FP32 residual has fallen by `delta` (0 < delta < 1) since the last
 * one, or when the FP32 recursion reports convergence. Convergence is declared only on the
 * FP64 residual (||b - A x|| <= opt->rtol ||b||). Unlike dg_refine_solve, no Krylov space is
 * restarted. opt->max_iters bounds the FP32 iterations. info: iters = FP32 iterations,
 * outer = updates, relres = FP64 relative residual. Errors as dg_refine_solve. */
dg_status dg_mixed_cg_solve(const dg_operator *op64, const dg_operator *op32, const double *b,
                            double *x, int nrhs, double delta, const dg_cg_options *opt,
                            dg_solve_info *info, void *stream);


/* y = A x for the FP64 scalar operator on the affine nx x ny x nz unit-cube mesh (the
 * same operator as dg_operator_create with vertices = NULL, DG_PEN_CONFIG penalty
 * alpha*k(k+1)/h_a, kappa = 1, one right-hand side), without any device allocation.
 * The paper has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code running inside a host application or framework that owns all device
 * memory through its own pool, and latency-critical loops that must not take the
 * implicit device synchronisation that cudaMalloc/cudaFree can cause. Instead of
 * operator-owned buffers it uses one file-scope device array of 32 MiB (reserved on
 * every GPU that loads libdg until the process exits) for the reference tables and the
 * apply's scratch; the caller passes x and y (device, 16-byte aligned, [ncell][(k+1)^3],
 * non-overlapping).
 * Limit: ncell * ((k+1)^3 + 24 (k+1)^2) * 8 bytes must fit in 32 MiB - 20 KiB (e.g.
 * 9356 cells at Q3); larger problems return DG_ERR_UNSUPPORTED without launching.
 * Set-up: the first call on a device, with that device current, looks up the array's
 * device address and uploads the reference tables of degrees 1..5 into it with one
 * synchronous copy; make that first call before any stream capture. Later calls on the
 * device only launch the apply's three kernels on `stream`. A cudaDeviceReset discards
 * the array and its tables, so the entry point must not be used on that device again
 * in the same process after a reset.
 * All calls share the array: calls that overlap on the GPU (different streams, or
 * concurrent host threads) race on it and must be ordered by the caller. Within one call
 * every scratch entry is written before it is read, so leftovers of earlier calls do no
 * harm. Errors: DG_ERR_INVALID_ARG (bad size, NULL, misaligned or overlapping x and y),
 * DG_ERR_UNSUPPORTED (degree > 5 or over the limit), DG_ERR_CUDA. */
dg_status dg_apply_affine_static(int nx, int ny, int nz, int degree, double c, double theta,
                                 double penalty_alpha, int dirichlet_mask, const double *x,
                                 double *y, void *stream);

/* Per-kernel timing for measurement harnesses. With enable != 0, every later apply on
 * this operator records CUDA events on its own stream before and after each of its
 * kernels (cell, face, back-projection). dg_operator_kernel_times waits for those events,
 * returns the summed milliseconds per kernel over the applies recorded since the last
 * call and their count, and starts a new accumulation. Errors: DG_ERR_INVALID_ARG,
 * DG_ERR_CUDA. */
dg_status dg_operator_profile(dg_operator *op, int enable);
dg_status dg_operator_kernel_times(dg_operator *op, double ms[3], int64_t *napplies);

/* Measured FMA throughput of this GPU for measurement harnesses (the paper reports its
 * operator throughput as a fraction of the machine's peak, Sec. 5): a kernel in which
 * every thread runs eight independent FMA chains in the given precision (DG_FP64 or
 * DG_FP32), one wave of blocks filling every SM, calibrated to about 50 ms per launch and
 * timed with CUDA events on `stream`; *tflops receives the best of three launches in
 * TFLOP/s (FMA = 2 flops). Allocates and frees a small output buffer; synchronises the
 * stream. Errors: DG_ERR_INVALID_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_measure_fma_peak(int precision, void *stream, double *tflops);

/* Measured tensor-core throughput for measurement harnesses, with the same protocol as
 * dg_measure_fma_peak: kind 0 = FP64 mma.sync m8n8k4 (DMMA), kind 1 = TF32 mma.sync
 * m16n8k8 with FP32 accumulation; every warp keeps four independent accumulations in
 * flight. kind 2 = DMMA and DFMA chains issued together by every warp (their combined
 * rate, which shows whether the two share one pipe). *tflops in TFLOP/s (one multiply-add = 2 flops). These decide whether the
 * batched 1D contractions of the sum factorisation (Sec. 2.2) could gain from the tensor
 * cores of this part. Errors: DG_ERR_INVALID_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_measure_mma_peak(int kind, void *stream, double *tflops);

/* Device-side faults recorded by kernels on the current device since the last clear
 * (bit mask in *faults, 0 if none): bit 0 = a wait of the persistent cellwise kernel for
 * its bulk copies into shared memory (x rows and brick-boundary neighbours, FP32 k = 2)
 * gave up after about one second; that launch stopped early and its output is invalid.
 * Synchronises with the device (it reads device memory). clear != 0 resets the mask.
 * Errors: DG_ERR_INVALID_ARG (faults NULL), DG_ERR_CUDA. */
dg_status dg_device_faults(int clear, unsigned *faults);

/* Reference-element tables the CUDA path uses (host, double), for inspection:
 * gauss_nodes/weights [m] on [0,1], gll_nodes [k+1], interp [m][k+1] (GLL Lagrange
 * basis at Gauss points), dcol [m][m] (derivative of the Gauss-point Lagrange basis at
 * the Gauss points), end_val[2][m], end_der[2][m] (that basis and its derivative at 0
 * and 1). Any output may be NULL. */
dg_status dg_reference_tables(int degree, int m, double *gauss_nodes, double *gauss_weights,
                              double *gll_nodes, double *interp, double *dcol,
                              double *end_val, double *end_der);

#ifdef __cplusplus
}
#endif
#endif
