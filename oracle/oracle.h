/*
 * Oracle for the matrix-free SIPG-DG operator of Kempf, Hess, Muething, Bastian,
 * "Automatic Code Generation for High-Performance Discontinuous Galerkin Methods on
 * Modern Architectures" (arXiv 1812.08075).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow CPU evaluation of the bilinear forms
 * of Eq. (diffreac_weak) (Sec. 5.2) and Eq. (stokes_weak) (Sec. 5.3), cell by cell and
 * face by face, with the full (non-factorised) tensor-product basis evaluated at every
 * Gauss point. It shares no code with the CUDA library and is used only by the tests,
 * the smoke check and the bench's CPU-baseline leg.
 *
 * Readings of the paper fixed here (the paper leaves them open):
 *   - local basis: Lagrange polynomials on the k+1 Gauss-Lobatto-Legendre points of
 *     [0,1] per direction (Sec. 2.1 says the basis choice is not important);
 *   - quadrature: m-point Gauss-Legendre per direction (Sec. 2.1, "1D rules");
 *   - DOF order in a cell: j0 + p*(j1 + p*j2), cells lexicographic, cell-major vector;
 *   - interior face normal from the lower-index cell T- to T+ (Sec. 2.1), jump
 *     [v] = v|T- - v|T+ (Sec. 5.2); boundary faces: jump = average = trace, outward n;
 *   - penalty: mode 0 gamma_F = alpha*k*(k+1)*n_a (h_a = 1/n_a across the face),
 *     mode 1 the paper's alpha*k*(k+d-1)*|F|/min(|T+|,|T-|) with measures by the same
 *     Gauss rule;
 *   - per-quadrature-point scalar kappa: volume [ncell][m^3], face [ncell][6][m^2]
 *     (each cell's own trace side, local faces -x,+x,-y,+y,-z,+z);
 *   - anisotropic degrees (Sec. 2.1's vector k, scalar problem): k_a per direction with
 *     k_a + 1 Gauss points; penalty mode 0 uses the degree along the face normal,
 *     gamma_F = alpha k_a (k_a + 1) n_a (the trace inverse inequality of a tensor-product
 *     polynomial scales with it), mode 1 likewise with k_a (k_a + d - 1);
 *   - Stokes: velocity Q_k x3 then pressure Q_{k-1}, vector [u: ncell x 3 x p^3 | p:
 *     ncell x k^3]; viscous block = scalar SIPG with kappa = mu, c = 0 on each component,
 *     face terms on interior and Dirichlet faces only.
 *
 * Parity unpinned: nothing in this file is unpinned; every routine is checked by the
 * CPU tests against closed forms, library routines, an independent Kronecker-product
 * construction (affine meshes), exactness identities and convergence rates.
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nx, ny, nz;
  int32_t k;              /* polynomial degree (velocity degree for Stokes) */
  int32_t m;              /* Gauss points per direction */
  int32_t pen_mode;       /* 0: alpha*k(k+1)/h_a, 1: paper's alpha*k(k+d-1)|F|/min|T| */
  int32_t dirichlet_mask; /* bit lf set: domain face lf (-x,+x,-y,+y,-z,+z) is Dirichlet */
  int32_t problem;        /* 0 scalar diffusion-reaction, 1 Stokes */
  double c;               /* reaction coefficient (scalar problem) */
  double mu;              /* viscosity (Stokes) */
  double theta;           /* -1 SIPG, 0 IIPG, +1 NIPG */
  double pen_alpha;
  const double *vertices; /* [(nx+1)(ny+1)(nz+1)][3] or NULL for the unit cube */
  const double *kappa_vol;  /* [ncell][m^3] or NULL (kappa = 1) */
  const double *kappa_face; /* [ncell][6][m^2] or NULL (kappa = 1) */
  int32_t kaxis[3];       /* anisotropic degrees (k_0, k_1, k_2), all >= 1, or all 0 for k in
                             every direction; anisotropic: scalar problem, cell DOFs
                             j0 + p0 (j1 + p1 j2) */
  int32_t maxis[3];       /* with kaxis: Gauss points per direction (m_0, m_1, m_2), 0 = k_a + 1.
                             kappa layouts then follow the per-direction counts:
                             kappa_vol [ncell][m0 m1 m2] (q0 + m0 (q1 + m1 q2)),
                             kappa_face [ncell][sum over lf of m_t1 m_t2], faces lf = 0..5 in
                             order, face points qs + m_t1 qt (t1 < t2 the tangential axes) */
  int32_t reserved;
} oracle_problem;

/* 1D rules on [0,1]. Return 0 on success. */
int oracle_gauss_rule(int m, double *nodes, double *weights);
int oracle_gll_nodes(int k, double *nodes);

/* Number of DOFs of the problem's vector. */
int64_t oracle_ndofs(const oracle_problem *pb);

/* y = A x (transpose = 0) or y = A^T x (transpose = 1). Returns 0 on success. */
int oracle_apply(const oracle_problem *pb, int transpose, const double *x, double *y);

/* y restricted to the listed cells: y_cells[i][:] = (A x) on cell cells[i]. Each listed
 * cell gathers its own volume term and its six faces' contributions to itself; the
 * loop over listed cells runs on nthreads OpenMP threads (<= 0: runtime default). */
int oracle_apply_cells(const oracle_problem *pb, int transpose, const double *x,
                       int64_t ncells, const int64_t *cells, double *y_cells, int nthreads);

/* Gradient of L = 0.5 ||A(kappa) x - b||^2 with respect to kappa given r = A x - b:
 * dk_vol[c][q] = r^T (dA/dkappa_vol[c][q]) x, dk_face[c][lf][q] likewise (scalar only). */
int oracle_dkappa(const oracle_problem *pb, const double *x, const double *r,
                  double *dk_vol, double *dk_face);

/* Data terms of Eq. (diffreac_weak) moved to the right-hand side (scalar problem):
 * F_i = (f, phi_i) + theta (g, n.kappa grad phi_i)_{Gamma_D} + gamma_F (g, phi_i)_{Gamma_D},
 * so that the residual is r = A u - F. f_vol: f at the volume Gauss points [ncell][m^3]
 * (NULL = 0); g_face: g at each cell's face Gauss points [ncell][6][m^2], read only on
 * Dirichlet boundary faces (NULL = 0). */
int oracle_rhs(const oracle_problem *pb, const double *f_vol, const double *g_face, double *F);

/* Semilinear reaction (scalar problem): mode 0: y = A w + beta (w^3, v), the residual
 * operator r(w); mode 1: y = A w + 3 beta (u0^2 w, v), its Jacobian action at u0. */
int oracle_semilinear(const oracle_problem *pb, double beta, int mode, const double *u0, const double *w,
                      double *y);

/* COO assembly of A from per-cell and per-face local matrices. Returns the number of
 * entries written, or -(needed) if cap is too small, or a value < -(1<<60) on error. */
int64_t oracle_assemble_coo(const oracle_problem *pb, int64_t cap, int64_t *rows,
                            int64_t *cols, double *vals);

#ifdef __cplusplus
}
#endif
#endif
