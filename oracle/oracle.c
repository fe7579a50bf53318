/*
 * Oracle: plain CPU evaluation of the SIPG-DG operator (TEST INFRASTRUCTURE ONLY).
 * See oracle.h for the readings of the paper it fixes. Every integral is a Gauss sum
 * with the full tensor-product basis evaluated point by point (no sum factorisation),
 * the geometry is the trilinear map of each cell's eight vertices (Sec. 2.1, mu_T).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OMAXP 8            /* up to degree 7 */
#define OMAXM 10
#define OMAXP3 (OMAXP * OMAXP * OMAXP)
#define OMAXL (3 * OMAXP3 + OMAXP3) /* Stokes local vector bound */

/* ------------------------------------------------------------------------------ */
/* 1D rules: Newton iteration on Legendre polynomials (three-term recurrence).     */
/* ------------------------------------------------------------------------------ */

/* P_n(t) and P_n'(t) on [-1,1] by the three-term recurrence. */
static void legendre(int n, long double t, long double *pn, long double *dpn) {
  long double p0 = 1.0L, p1 = t;
  if (n == 0) { *pn = 1.0L; *dpn = 0.0L; return; }
  for (int j = 2; j <= n; ++j) {
    long double p2 = ((2.0L * j - 1.0L) * t * p1 - (j - 1.0L) * p0) / (long double)j;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  /* derivative from (1-t^2) P_n' = n (P_{n-1} - t P_n) */
  *dpn = (long double)n * (p0 - t * p1) / (1.0L - t * t);
}

int oracle_gauss_rule(int m, double *nodes, double *weights) {
  if (m < 1 || m > OMAXM) return 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < m; ++i) {
    /* initial guess for the i-th root (descending), then Newton */
    long double t = cosl(pi * (i + 0.75L) / (m + 0.5L));
    for (int it = 0; it < 100; ++it) {
      long double p, dp;
      legendre(m, t, &p, &dp);
      long double dt = p / dp;
      t -= dt;
      if (fabsl(dt) < 1e-19L) break;
    }
    long double p, dp;
    legendre(m, t, &p, &dp);
    long double w = 2.0L / ((1.0L - t * t) * dp * dp);
    /* ascending order on [0,1] */
    nodes[m - 1 - i] = (double)((1.0L + t) / 2.0L);
    weights[m - 1 - i] = (double)(w / 2.0L);
  }
  return 0;
}

int oracle_gll_nodes(int k, double *nodes) {
  if (k < 1 || k + 1 > OMAXP) return 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  nodes[0] = 0.0;
  nodes[k] = 1.0;
  /* interior GLL points are the roots of P_k'; Newton with P_k'' from Legendre's ODE */
  for (int i = 1; i < k; ++i) {
    long double t = -cosl(pi * i / (long double)k);
    for (int it = 0; it < 100; ++it) {
      long double p, dp;
      legendre(k, t, &p, &dp);
      long double d2p = (2.0L * t * dp - (long double)k * (k + 1) * p) / (1.0L - t * t);
      long double dt = dp / d2p;
      t -= dt;
      if (fabsl(dt) < 1e-19L) break;
    }
    nodes[i] = (double)((1.0L + t) / 2.0L);
  }
  return 0;
}

/* ------------------------------------------------------------------------------ */
/* Lagrange basis on a node set, evaluated by the product formula.                 */
/* ------------------------------------------------------------------------------ */

static void lagrange_1d(int n, const double *z, double t, double *val, double *der) {
  for (int j = 0; j < n; ++j) {
    long double v = 1.0L;
    for (int i = 0; i < n; ++i)
      if (i != j) v *= ((long double)t - z[i]) / ((long double)z[j] - z[i]);
    long double d = 0.0L;
    for (int l = 0; l < n; ++l) {
      if (l == j) continue;
      long double term = 1.0L / ((long double)z[j] - z[l]);
      for (int i = 0; i < n; ++i)
        if (i != j && i != l) term *= ((long double)t - z[i]) / ((long double)z[j] - z[i]);
      d += term;
    }
    val[j] = (double)v;
    der[j] = (double)d;
  }
}

/* ------------------------------------------------------------------------------ */
/* Problem context                                                                 */
/* ------------------------------------------------------------------------------ */

typedef struct {
  const oracle_problem *pb;
  int n[3];
  int p, m, pp;            /* basis points, quad points, pressure basis points (isotropic) */
  int P3, PP3, L;          /* local sizes */
  int64_t ncell;
  double s[OMAXM], w[OMAXM];
  double zv[OMAXP], zp[OMAXP];
  /* per direction (equal to the above unless the degrees are anisotropic) */
  int aniso;
  int ka[3], pa[3], ma[3];
  double sa[3][OMAXM], wa[3][OMAXM], za[3][OMAXP];
  /* kappa layouts: volume points per cell; face points per cell and face offsets */
  int nqv, nqf, fo[7];
} octx;

static void tangential_axes(int a, int *t1, int *t2);

static int ctx_init(octx *o, const oracle_problem *pb) {
  memset(o, 0, sizeof(*o));
  o->pb = pb;
  if (pb->nx < 1 || pb->ny < 1 || pb->nz < 1) return 1;
  if (pb->k < 1 || pb->k + 1 > OMAXP || pb->m < 1 || pb->m > OMAXM) return 1;
  if (pb->problem != 0 && pb->problem != 1) return 1;
  if (pb->problem == 1 && pb->k < 2) return 1;
  o->n[0] = pb->nx; o->n[1] = pb->ny; o->n[2] = pb->nz;
  o->p = pb->k + 1;
  o->m = pb->m;
  o->P3 = o->p * o->p * o->p;
  o->ncell = (int64_t)pb->nx * pb->ny * pb->nz;
  if (oracle_gauss_rule(o->m, o->s, o->w)) return 1;
  if (oracle_gll_nodes(pb->k, o->zv)) return 1;
  o->aniso = pb->kaxis[0] != 0 || pb->kaxis[1] != 0 || pb->kaxis[2] != 0;
  for (int d = 0; d < 3; ++d) {
    if (o->aniso) {
      const int kd = pb->kaxis[d];
      const int md = pb->maxis[d] ? pb->maxis[d] : kd + 1;
      if (kd < 1 || kd + 1 > OMAXP || md < 1 || md > OMAXM || pb->problem != 0) return 1;
      o->ka[d] = kd;
      o->pa[d] = kd + 1;
      o->ma[d] = md;
      if (oracle_gauss_rule(o->ma[d], o->sa[d], o->wa[d])) return 1;
      if (oracle_gll_nodes(kd, o->za[d])) return 1;
    } else {
      o->ka[d] = pb->k;
      o->pa[d] = o->p;
      o->ma[d] = o->m;
      memcpy(o->sa[d], o->s, sizeof(o->s));
      memcpy(o->wa[d], o->w, sizeof(o->w));
      memcpy(o->za[d], o->zv, sizeof(o->zv));
    }
  }
  if (o->aniso) o->P3 = o->pa[0] * o->pa[1] * o->pa[2];
  o->nqv = o->ma[0] * o->ma[1] * o->ma[2];
  o->fo[0] = 0;
  for (int lf = 0; lf < 6; ++lf) {
    int t1, t2;
    tangential_axes(lf >> 1, &t1, &t2);
    o->fo[lf + 1] = o->fo[lf] + o->ma[t1] * o->ma[t2];
  }
  o->nqf = o->fo[6];
  if (pb->problem == 1) {
    o->pp = pb->k; /* pressure degree k-1 */
    if (oracle_gll_nodes(pb->k - 1, o->zp)) return 1;
    o->PP3 = o->pp * o->pp * o->pp;
    o->L = 3 * o->P3 + o->PP3;
  } else {
    o->L = o->P3;
  }
  return 0;
}

int64_t oracle_ndofs(const oracle_problem *pb) {
  octx o;
  if (ctx_init(&o, pb)) return -1;
  return o.ncell * o.L;
}

static void cell_coords(const octx *o, int64_t c, int cc[3]) {
  cc[0] = (int)(c % o->n[0]);
  cc[1] = (int)((c / o->n[0]) % o->n[1]);
  cc[2] = (int)(c / ((int64_t)o->n[0] * o->n[1]));
}

static int64_t cell_index(const octx *o, const int cc[3]) {
  return cc[0] + (int64_t)o->n[0] * (cc[1] + (int64_t)o->n[1] * cc[2]);
}

static void cell_vertices(const octx *o, int64_t c, double V[8][3]) {
  int cc[3];
  cell_coords(o, c, cc);
  for (int a = 0; a < 8; ++a) {
    int i = cc[0] + (a & 1), j = cc[1] + ((a >> 1) & 1), l = cc[2] + ((a >> 2) & 1);
    if (o->pb->vertices) {
      int64_t v = i + (int64_t)(o->n[0] + 1) * (j + (int64_t)(o->n[1] + 1) * l);
      for (int d = 0; d < 3; ++d) V[a][d] = o->pb->vertices[3 * v + d];
    } else {
      V[a][0] = (double)i / o->n[0];
      V[a][1] = (double)j / o->n[1];
      V[a][2] = (double)l / o->n[2];
    }
  }
}

/* Jacobian J[i][d] = d x_i / d xi_d of the trilinear map through the 8 vertices. */
static void map_jacobian(double V[8][3], const double xi[3], double J[3][3]) {
  memset(J, 0, 9 * sizeof(double));
  for (int a = 0; a < 8; ++a) {
    int b[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
    double f[3], df[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = b[d] ? xi[d] : 1.0 - xi[d];
      df[d] = b[d] ? 1.0 : -1.0;
    }
    double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) J[i][d] += dN[d] * V[a][i];
  }
}

static double det3(double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static void inv3(double J[3][3], double det, double Ji[3][3]) {
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

/* Full tensor-product basis on node set z (n per direction) at reference point xi:
 * phi[j] and physical gradients g[j] = J^{-T} grad_ref phi_j (Ji may be NULL: values only). */
static void basis3d(int n, const double *z, const double xi[3], double Ji[3][3],
                    double *phi, double (*g)[3]) {
  double v[3][OMAXP], dv[3][OMAXP];
  for (int d = 0; d < 3; ++d) lagrange_1d(n, z, xi[d], v[d], dv[d]);
  int j = 0;
  for (int j2 = 0; j2 < n; ++j2)
    for (int j1 = 0; j1 < n; ++j1)
      for (int j0 = 0; j0 < n; ++j0, ++j) {
        phi[j] = v[0][j0] * v[1][j1] * v[2][j2];
        if (g) {
          double gr[3] = {dv[0][j0] * v[1][j1] * v[2][j2], v[0][j0] * dv[1][j1] * v[2][j2],
                          v[0][j0] * v[1][j1] * dv[2][j2]};
          for (int i = 0; i < 3; ++i) g[j][i] = Ji[0][i] * gr[0] + Ji[1][i] * gr[1] + Ji[2][i] * gr[2];
        }
      }
}

/* basis3d with its own node set per direction: pa[d] nodes za[d] (anisotropic degrees). */
static void basis3d_axes(const int pa[3], const double za[3][OMAXP], const double xi[3], double Ji[3][3],
                         double *phi, double (*g)[3]) {
  double v[3][OMAXP], dv[3][OMAXP];
  for (int d = 0; d < 3; ++d) lagrange_1d(pa[d], za[d], xi[d], v[d], dv[d]);
  int j = 0;
  for (int j2 = 0; j2 < pa[2]; ++j2)
    for (int j1 = 0; j1 < pa[1]; ++j1)
      for (int j0 = 0; j0 < pa[0]; ++j0, ++j) {
        phi[j] = v[0][j0] * v[1][j1] * v[2][j2];
        if (g) {
          double gr[3] = {dv[0][j0] * v[1][j1] * v[2][j2], v[0][j0] * dv[1][j1] * v[2][j2],
                          v[0][j0] * v[1][j1] * dv[2][j2]};
          for (int i = 0; i < 3; ++i) g[j][i] = Ji[0][i] * gr[0] + Ji[1][i] * gr[1] + Ji[2][i] * gr[2];
        }
      }
}

/* Measures |T| and |F| by the same Gauss rule (penalty mode 1). */
static double cell_measure(const octx *o, int64_t c) {
  double V[8][3], J[3][3], xi[3], vol = 0.0;
  cell_vertices(o, c, V);
  for (int q2 = 0; q2 < o->ma[2]; ++q2)
    for (int q1 = 0; q1 < o->ma[1]; ++q1)
      for (int q0 = 0; q0 < o->ma[0]; ++q0) {
        xi[0] = o->sa[0][q0]; xi[1] = o->sa[1][q1]; xi[2] = o->sa[2][q2];
        map_jacobian(V, xi, J);
        vol += o->wa[0][q0] * o->wa[1][q1] * o->wa[2][q2] * det3(J);
      }
  return vol;
}

static void tangential_axes(int a, int *t1, int *t2) {
  *t1 = (a == 0) ? 1 : 0;
  *t2 = (a == 2) ? 1 : 2;
}

/* Area vector at a face point of cell c, local face lf = 2a+side: cross product of the
 * two tangential columns of J, oriented towards +xi_a for side 1 and -xi_a for side 0. */
static void face_area_vector(double J[3][3], int a, int side, double nv[3]) {
  int t1, t2;
  tangential_axes(a, &t1, &t2);
  double u[3] = {J[0][t1], J[1][t1], J[2][t1]}, v[3] = {J[0][t2], J[1][t2], J[2][t2]};
  nv[0] = u[1] * v[2] - u[2] * v[1];
  nv[1] = u[2] * v[0] - u[0] * v[2];
  nv[2] = u[0] * v[1] - u[1] * v[0];
  double along = nv[0] * J[0][a] + nv[1] * J[1][a] + nv[2] * J[2][a];
  double want = side ? 1.0 : -1.0;
  if (along * want < 0) { nv[0] = -nv[0]; nv[1] = -nv[1]; nv[2] = -nv[2]; }
}

static double face_measure(const octx *o, int64_t c, int a, int side) {
  double V[8][3], J[3][3], xi[3], nv[3], area = 0.0;
  int t1, t2;
  tangential_axes(a, &t1, &t2);
  cell_vertices(o, c, V);
  for (int qt = 0; qt < o->ma[t2]; ++qt)
    for (int qs = 0; qs < o->ma[t1]; ++qs) {
      xi[a] = side ? 1.0 : 0.0; xi[t1] = o->sa[t1][qs]; xi[t2] = o->sa[t2][qt];
      map_jacobian(V, xi, J);
      face_area_vector(J, a, side, nv);
      area += o->wa[t1][qs] * o->wa[t2][qt] * sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    }
  return area;
}

/* gamma_F, Sec. 5.2 (mode 1) or alpha*k(k+1)/h_a with h_a = 1/n_a (mode 0). */
static double penalty(const octx *o, int a, int64_t cm, int sidem, int64_t cp) {
  int k = o->ka[a];  /* the degree along the face normal (k in every direction if isotropic) */
  if (o->pb->pen_mode == 0) return o->pb->pen_alpha * k * (k + 1) * (double)o->n[a];
  double F = face_measure(o, cm, a, sidem);
  double T = cell_measure(o, cm);
  if (cp >= 0) {
    double Tp = cell_measure(o, cp);
    if (Tp < T) T = Tp;
  }
  return o->pb->pen_alpha * k * (k + 3 - 1) * F / T;
}

/* ------------------------------------------------------------------------------ */
/* Local integrals                                                                  */
/* ------------------------------------------------------------------------------ */

/* Volume term of Eq. (diffreac_weak): ye += int_T kappa grad u . grad v + c u v. */
static void vol_scalar(const octx *o, int64_t c, const double *xe, double *ye) {
  double V[8][3], J[3][3], Ji[3][3], xi[3];
  static __thread double phi[OMAXP3], g[OMAXP3][3];
  const int P3 = o->P3;
  cell_vertices(o, c, V);
  for (int q2 = 0; q2 < o->ma[2]; ++q2)
    for (int q1 = 0; q1 < o->ma[1]; ++q1)
      for (int q0 = 0; q0 < o->ma[0]; ++q0) {
        xi[0] = o->sa[0][q0]; xi[1] = o->sa[1][q1]; xi[2] = o->sa[2][q2];
        double W = o->wa[0][q0] * o->wa[1][q1] * o->wa[2][q2];
        map_jacobian(V, xi, J);
        double dJ = det3(J);
        inv3(J, dJ, Ji);
        basis3d_axes(o->pa, o->za, xi, Ji, phi, g);
        double u = 0, gu[3] = {0, 0, 0};
        for (int j = 0; j < P3; ++j) {
          u += xe[j] * phi[j];
          for (int i = 0; i < 3; ++i) gu[i] += xe[j] * g[j][i];
        }
        int q = q0 + o->ma[0] * (q1 + o->ma[1] * q2);
        double kap = o->pb->kappa_vol ? o->pb->kappa_vol[c * o->nqv + q] : 1.0;
        double cr = o->pb->c;
        for (int i = 0; i < P3; ++i)
          ye[i] += W * dJ * (kap * (gu[0] * g[i][0] + gu[1] * g[i][1] + gu[2] * g[i][2]) + cr * u * phi[i]);
      }
}

/* Trace data of one side of a face at face point (qs, qt). */
typedef struct {
  double phi[OMAXP3];     /* basis values */
  double dn[OMAXP3];      /* grad phi . n (physical) */
  double g[OMAXP3][3];    /* physical gradients */
  double ppsi[OMAXP3];    /* pressure basis values (Stokes) */
} side_data;

/* Evaluate one side: geometry of cell c at local face (a, side), face point (qs, qt),
 * with the unit normal n supplied (or computed when nrm_in is NULL). */
static void side_eval(const octx *o, int64_t c, int a, int side, int qs, int qt,
                      const double *nrm_in, double nrm_out[3], double *ds_out, side_data *sd) {
  double V[8][3], J[3][3], Ji[3][3], xi[3];
  int t1, t2;
  tangential_axes(a, &t1, &t2);
  cell_vertices(o, c, V);
  xi[a] = side ? 1.0 : 0.0; xi[t1] = o->sa[t1][qs]; xi[t2] = o->sa[t2][qt];
  map_jacobian(V, xi, J);
  double dJ = det3(J);
  inv3(J, dJ, Ji);
  if (!nrm_in) {
    double nv[3];
    face_area_vector(J, a, side, nv);
    double ds = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int i = 0; i < 3; ++i) nrm_out[i] = nv[i] / ds;
    *ds_out = ds;
    nrm_in = nrm_out;
  }
  basis3d_axes(o->pa, o->za, xi, Ji, sd->phi, sd->g);
  for (int j = 0; j < o->P3; ++j)
    sd->dn[j] = sd->g[j][0] * nrm_in[0] + sd->g[j][1] * nrm_in[1] + sd->g[j][2] * nrm_in[2];
  if (o->pb->problem == 1) basis3d(o->pp, o->zp, xi, NULL, sd->ppsi, NULL);
}

static double kappa_face_at(const octx *o, int64_t c, int lf, int qs, int qt) {
  if (!o->pb->kappa_face) return 1.0;
  int t1, t2;
  tangential_axes(lf >> 1, &t1, &t2);
  return o->pb->kappa_face[c * o->nqf + o->fo[lf] + qs + o->ma[t1] * qt];
}

/* Face terms of Eq. (diffreac_weak) on one face. cp < 0: boundary face of cm at
 * (a, sidem). sc multiplies -n.{kappa grad u}[v]'s flux (forward: -1) and ss the
 * symmetry term [u] n.{kappa grad v} (forward: theta); the transpose a(v,u) swaps them.
 * ym/yp accumulate the local residual of the two sides (only ym on a boundary face). */
static void face_scalar(const octx *o, int a, int64_t cm, int sidem, int64_t cp,
                        const double *xm, const double *xp, double *ym, double *yp,
                        double sc, double ss) {
  static __thread side_data dm, dp;
  const int P3 = o->P3;
  int t1, t2;
  tangential_axes(a, &t1, &t2);
  double gam = penalty(o, a, cm, sidem, cp);
  for (int qt = 0; qt < o->ma[t2]; ++qt)
    for (int qs = 0; qs < o->ma[t1]; ++qs) {
      double n[3], ds;
      side_eval(o, cm, a, sidem, qs, qt, NULL, n, &ds, &dm);
      double W = o->wa[t1][qs] * o->wa[t2][qt] * ds;
      double um = 0, gnm = 0;
      for (int j = 0; j < P3; ++j) { um += xm[j] * dm.phi[j]; gnm += xm[j] * dm.dn[j]; }
      double km = kappa_face_at(o, cm, 2 * a + sidem, qs, qt);
      if (cp >= 0) {
        double dummy[3], dsd;
        side_eval(o, cp, a, 0, qs, qt, n, dummy, &dsd, &dp);
        double up = 0, gnp = 0;
        for (int j = 0; j < P3; ++j) { up += xp[j] * dp.phi[j]; gnp += xp[j] * dp.dn[j]; }
        double kp = kappa_face_at(o, cp, 2 * a, qs, qt);
        double jump = um - up;
        double avg = 0.5 * (km * gnm + kp * gnp);
        double tv = sc * avg + gam * jump;
        for (int i = 0; i < P3; ++i) {
          ym[i] += W * (tv * dm.phi[i] + ss * jump * 0.5 * km * dm.dn[i]);
          yp[i] += W * (-tv * dp.phi[i] + ss * jump * 0.5 * kp * dp.dn[i]);
        }
      } else {
        double tv = sc * km * gnm + gam * um;
        for (int i = 0; i < P3; ++i) ym[i] += W * (tv * dm.phi[i] + ss * um * km * dm.dn[i]);
      }
    }
}

/* Volume terms of Eq. (stokes_weak): viscous (mu grad u_c, grad v_c), -(p, div v),
 * -(div u, q). Local vector [u0|u1|u2|p]. */
static void vol_stokes(const octx *o, int64_t c, const double *xe, double *ye) {
  double V[8][3], J[3][3], Ji[3][3], xi[3];
  static __thread double phi[OMAXP3], g[OMAXP3][3], psi[OMAXP3];
  const int P3 = o->P3, PP3 = o->PP3, m = o->m;
  const double mu = o->pb->mu;
  cell_vertices(o, c, V);
  for (int q2 = 0; q2 < m; ++q2)
    for (int q1 = 0; q1 < m; ++q1)
      for (int q0 = 0; q0 < m; ++q0) {
        xi[0] = o->s[q0]; xi[1] = o->s[q1]; xi[2] = o->s[q2];
        double W = o->w[q0] * o->w[q1] * o->w[q2];
        map_jacobian(V, xi, J);
        double dJ = det3(J);
        inv3(J, dJ, Ji);
        basis3d(o->p, o->zv, xi, Ji, phi, g);
        basis3d(o->pp, o->zp, xi, NULL, psi, NULL);
        double gu[3][3] = {{0}};
        for (int cc = 0; cc < 3; ++cc)
          for (int j = 0; j < P3; ++j)
            for (int i = 0; i < 3; ++i) gu[cc][i] += xe[cc * P3 + j] * g[j][i];
        double pr = 0;
        for (int l = 0; l < PP3; ++l) pr += xe[3 * P3 + l] * psi[l];
        double div = gu[0][0] + gu[1][1] + gu[2][2];
        for (int cc = 0; cc < 3; ++cc)
          for (int i = 0; i < P3; ++i)
            ye[cc * P3 + i] += W * dJ *
                (mu * (gu[cc][0] * g[i][0] + gu[cc][1] * g[i][1] + gu[cc][2] * g[i][2]) - pr * g[i][cc]);
        for (int l = 0; l < PP3; ++l) ye[3 * P3 + l] += W * dJ * (-div * psi[l]);
      }
}

/* Face terms of Eq. (stokes_weak) on interior and Dirichlet faces: viscous SIPG per
 * component (kappa = mu), ({p}, [v].n) and ([u].n, {q}). */
static void face_stokes(const octx *o, int a, int64_t cm, int sidem, int64_t cp,
                        const double *xm, const double *xp, double *ym, double *yp,
                        double sc, double ss) {
  static __thread side_data dm, dp;
  const int P3 = o->P3, PP3 = o->PP3, m = o->m;
  const double mu = o->pb->mu;
  double gam = penalty(o, a, cm, sidem, cp);
  for (int qt = 0; qt < m; ++qt)
    for (int qs = 0; qs < m; ++qs) {
      double n[3], ds;
      side_eval(o, cm, a, sidem, qs, qt, NULL, n, &ds, &dm);
      double W = o->w[qs] * o->w[qt] * ds;
      double um[3] = {0, 0, 0}, gnm[3] = {0, 0, 0}, pm = 0;
      for (int cc = 0; cc < 3; ++cc)
        for (int j = 0; j < P3; ++j) { um[cc] += xm[cc * P3 + j] * dm.phi[j]; gnm[cc] += xm[cc * P3 + j] * dm.dn[j]; }
      for (int l = 0; l < PP3; ++l) pm += xm[3 * P3 + l] * dm.ppsi[l];
      if (cp >= 0) {
        double dummy[3], dsd;
        side_eval(o, cp, a, 0, qs, qt, n, dummy, &dsd, &dp);
        double up[3] = {0, 0, 0}, gnp[3] = {0, 0, 0}, pp = 0;
        for (int cc = 0; cc < 3; ++cc)
          for (int j = 0; j < P3; ++j) { up[cc] += xp[cc * P3 + j] * dp.phi[j]; gnp[cc] += xp[cc * P3 + j] * dp.dn[j]; }
        for (int l = 0; l < PP3; ++l) pp += xp[3 * P3 + l] * dp.ppsi[l];
        double pavg = 0.5 * (pm + pp);
        double jn = 0;
        for (int cc = 0; cc < 3; ++cc) jn += (um[cc] - up[cc]) * n[cc];
        for (int cc = 0; cc < 3; ++cc) {
          double jump = um[cc] - up[cc];
          double avg = 0.5 * mu * (gnm[cc] + gnp[cc]);
          double tv = sc * avg + gam * jump;
          for (int i = 0; i < P3; ++i) {
            ym[cc * P3 + i] += W * (tv * dm.phi[i] + ss * jump * 0.5 * mu * dm.dn[i] + pavg * n[cc] * dm.phi[i]);
            yp[cc * P3 + i] += W * (-tv * dp.phi[i] + ss * jump * 0.5 * mu * dp.dn[i] - pavg * n[cc] * dp.phi[i]);
          }
        }
        for (int l = 0; l < PP3; ++l) {
          ym[3 * P3 + l] += W * 0.5 * jn * dm.ppsi[l];
          yp[3 * P3 + l] += W * 0.5 * jn * dp.ppsi[l];
        }
      } else {
        double jn = um[0] * n[0] + um[1] * n[1] + um[2] * n[2];
        for (int cc = 0; cc < 3; ++cc) {
          double tv = sc * mu * gnm[cc] + gam * um[cc];
          for (int i = 0; i < P3; ++i)
            ym[cc * P3 + i] += W * (tv * dm.phi[i] + ss * um[cc] * mu * dm.dn[i] + pm * n[cc] * dm.phi[i]);
        }
        for (int l = 0; l < PP3; ++l) ym[3 * P3 + l] += W * jn * dm.ppsi[l];
      }
    }
}

/* ------------------------------------------------------------------------------ */
/* Gather / scatter of local vectors                                                */
/* ------------------------------------------------------------------------------ */

static void gather(const octx *o, int64_t c, const double *x, double *xe) {
  if (o->pb->problem == 0) {
    memcpy(xe, x + c * o->P3, o->P3 * sizeof(double));
  } else {
    memcpy(xe, x + c * 3 * o->P3, 3 * o->P3 * sizeof(double));
    memcpy(xe + 3 * o->P3, x + o->ncell * 3 * o->P3 + c * o->PP3, o->PP3 * sizeof(double));
  }
}

static void scatter_add(const octx *o, int64_t c, const double *ye, double *y) {
  if (o->pb->problem == 0) {
    for (int i = 0; i < o->P3; ++i) y[c * o->P3 + i] += ye[i];
  } else {
    for (int i = 0; i < 3 * o->P3; ++i) y[c * 3 * o->P3 + i] += ye[i];
    for (int i = 0; i < o->PP3; ++i) y[o->ncell * 3 * o->P3 + c * o->PP3 + i] += ye[3 * o->P3 + i];
  }
}

static void vol_local(const octx *o, int64_t c, const double *xe, double *ye) {
  if (o->pb->problem == 0) vol_scalar(o, c, xe, ye);
  else vol_stokes(o, c, xe, ye);
}

static void face_local(const octx *o, int a, int64_t cm, int sidem, int64_t cp, const double *xm,
                       const double *xp, double *ym, double *yp, int transpose) {
  double sc = -1.0, ss = o->pb->theta;
  if (transpose) { sc = o->pb->theta; ss = -1.0; }
  if (o->pb->problem == 0) face_scalar(o, a, cm, sidem, cp, xm, xp, ym, yp, sc, ss);
  else face_stokes(o, a, cm, sidem, cp, xm, xp, ym, yp, sc, ss);
}

/* Enumerate faces of axis a by (f, i1, i2): f in [0, n_a] is the position along a,
 * (i1, i2) the cell position along the tangential axes t1 < t2. Fills the cells on
 * both sides (-1 where absent). */
static void face_cells(const octx *o, int a, int f, int i1, int i2, int64_t *cm, int64_t *cp) {
  int t1, t2;
  tangential_axes(a, &t1, &t2);
  int cc[3];
  cc[t1] = i1; cc[t2] = i2;
  *cm = -1; *cp = -1;
  if (f > 0) { cc[a] = f - 1; *cm = cell_index(o, cc); }
  if (f < o->n[a]) { cc[a] = f; *cp = cell_index(o, cc); }
}

/* ------------------------------------------------------------------------------ */
/* Public entry points                                                              */
/* ------------------------------------------------------------------------------ */

int oracle_apply(const oracle_problem *pb, int transpose, const double *x, double *y) {
  octx o;
  if (ctx_init(&o, pb)) return 1;
  const int L = o.L;
  double *xe = malloc(sizeof(double) * 4 * L);
  if (!xe) return 2;
  double *ye = xe + L, *xe2 = xe + 2 * L, *ye2 = xe + 3 * L;
  memset(y, 0, sizeof(double) * o.ncell * L);
  for (int64_t c = 0; c < o.ncell; ++c) {
    gather(&o, c, x, xe);
    memset(ye, 0, sizeof(double) * L);
    vol_local(&o, c, xe, ye);
    scatter_add(&o, c, ye, y);
  }
  for (int a = 0; a < 3; ++a) {
    int t1, t2;
    tangential_axes(a, &t1, &t2);
    for (int i2 = 0; i2 < o.n[t2]; ++i2)
      for (int i1 = 0; i1 < o.n[t1]; ++i1)
        for (int f = 0; f <= o.n[a]; ++f) {
          int64_t cm, cp;
          face_cells(&o, a, f, i1, i2, &cm, &cp);
          memset(ye, 0, sizeof(double) * L);
          memset(ye2, 0, sizeof(double) * L);
          if (cm >= 0 && cp >= 0) {
            gather(&o, cm, x, xe);
            gather(&o, cp, x, xe2);
            face_local(&o, a, cm, 1, cp, xe, xe2, ye, ye2, transpose);
            scatter_add(&o, cm, ye, y);
            scatter_add(&o, cp, ye2, y);
          } else {
            int64_t cb = cm >= 0 ? cm : cp;
            int side = cm >= 0 ? 1 : 0;
            if (!((pb->dirichlet_mask >> (2 * a + side)) & 1)) continue;
            gather(&o, cb, x, xe);
            face_local(&o, a, cb, side, -1, xe, NULL, ye, NULL, transpose);
            scatter_add(&o, cb, ye, y);
          }
        }
  }
  free(xe);
  return 0;
}

/* Contribution of all integrals to the local residual of one cell (gather form). */
static void cell_gather(const octx *o, int64_t c, const double *x, int transpose, double *yc,
                        double *xe, double *xe2, double *tmp, double *tmp2) {
  const int L = o->L;
  memset(yc, 0, sizeof(double) * L);
  gather(o, c, x, xe);
  vol_local(o, c, xe, yc);
  int cc[3];
  cell_coords(o, c, cc);
  for (int a = 0; a < 3; ++a)
    for (int side = 0; side < 2; ++side) {
      int nb[3] = {cc[0], cc[1], cc[2]};
      nb[a] += side ? 1 : -1;
      memset(tmp, 0, sizeof(double) * L);
      memset(tmp2, 0, sizeof(double) * L);
      if (nb[a] < 0 || nb[a] >= o->n[a]) {
        if (!((o->pb->dirichlet_mask >> (2 * a + side)) & 1)) continue;
        face_local(o, a, c, side, -1, xe, NULL, tmp, NULL, transpose);
        for (int i = 0; i < L; ++i) yc[i] += tmp[i];
      } else {
        int64_t n = cell_index(o, nb);
        gather(o, n, x, xe2);
        if (side == 1) {
          face_local(o, a, c, 1, n, xe, xe2, tmp, tmp2, transpose);
          for (int i = 0; i < L; ++i) yc[i] += tmp[i];
        } else {
          face_local(o, a, n, 1, c, xe2, xe, tmp2, tmp, transpose);
          for (int i = 0; i < L; ++i) yc[i] += tmp[i];
        }
      }
    }
}

int oracle_apply_cells(const oracle_problem *pb, int transpose, const double *x,
                       int64_t ncells, const int64_t *cells, double *y_cells, int nthreads) {
  octx o;
  if (ctx_init(&o, pb)) return 1;
  for (int64_t i = 0; i < ncells; ++i)
    if (cells[i] < 0 || cells[i] >= o.ncell) return 1;
  const int L = o.L;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    double *buf = malloc(sizeof(double) * 4 * L);
    if (!buf) {
#pragma omp atomic write
      err = 2;
    } else {
#pragma omp for schedule(dynamic, 4)
      for (int64_t i = 0; i < ncells; ++i)
        cell_gather(&o, cells[i], x, transpose, y_cells + i * L, buf, buf + L, buf + 2 * L, buf + 3 * L);
      free(buf);
    }
  }
  return err;
}

int oracle_dkappa(const oracle_problem *pb, const double *x, const double *r,
                  double *dk_vol, double *dk_face) {
  octx o;
  if (ctx_init(&o, pb) || pb->problem != 0 || o.aniso) return 1;
  const int P3 = o.P3, m = o.m, m2 = m * m, m3 = m * m * m;
  static __thread side_data dm, dp;
  double *phi = malloc(sizeof(double) * P3 * 4);
  if (!phi) return 2;
  double (*g)[3] = (double (*)[3])(phi + P3);
  /* volume: d/dkappa_q of int kappa grad x . grad r = W detJ grad x . grad r at q */
  for (int64_t c = 0; c < o.ncell; ++c) {
    double V[8][3], J[3][3], Ji[3][3], xi[3];
    cell_vertices(&o, c, V);
    for (int q2 = 0; q2 < m; ++q2)
      for (int q1 = 0; q1 < m; ++q1)
        for (int q0 = 0; q0 < m; ++q0) {
          xi[0] = o.s[q0]; xi[1] = o.s[q1]; xi[2] = o.s[q2];
          double W = o.w[q0] * o.w[q1] * o.w[q2];
          map_jacobian(V, xi, J);
          double dJ = det3(J);
          inv3(J, dJ, Ji);
          basis3d(o.p, o.zv, xi, Ji, phi, g);
          double gx[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
          for (int j = 0; j < P3; ++j)
            for (int i = 0; i < 3; ++i) {
              gx[i] += x[c * P3 + j] * g[j][i];
              gr[i] += r[c * P3 + j] * g[j][i];
            }
          dk_vol[c * m3 + q0 + m * (q1 + m * q2)] = W * dJ * (gx[0] * gr[0] + gx[1] * gr[1] + gx[2] * gr[2]);
        }
  }
  free(phi);
  /* faces: kappa^s enters -n.{kappa grad x}[r] + theta [x] n.{kappa grad r} with
   * weight 1/2 on interior faces and 1 on Dirichlet faces */
  memset(dk_face, 0, sizeof(double) * o.ncell * 6 * m2);
  const double th = pb->theta;
  for (int a = 0; a < 3; ++a) {
    int t1, t2;
    tangential_axes(a, &t1, &t2);
    for (int i2 = 0; i2 < o.n[t2]; ++i2)
      for (int i1 = 0; i1 < o.n[t1]; ++i1)
        for (int f = 0; f <= o.n[a]; ++f) {
          int64_t cm, cp;
          face_cells(&o, a, f, i1, i2, &cm, &cp);
          int bnd = !(cm >= 0 && cp >= 0);
          int64_t c0 = cm >= 0 ? cm : cp;
          int side0 = cm >= 0 ? 1 : 0;
          if (bnd && !((pb->dirichlet_mask >> (2 * a + side0)) & 1)) continue;
          for (int qt = 0; qt < m; ++qt)
            for (int qs = 0; qs < m; ++qs) {
              double n[3], ds;
              side_eval(&o, c0, a, side0, qs, qt, NULL, n, &ds, &dm);
              double W = o.w[qs] * o.w[qt] * ds;
              double xm = 0, rm = 0, gxm = 0, grm = 0;
              for (int j = 0; j < P3; ++j) {
                xm += x[c0 * P3 + j] * dm.phi[j]; rm += r[c0 * P3 + j] * dm.phi[j];
                gxm += x[c0 * P3 + j] * dm.dn[j]; grm += r[c0 * P3 + j] * dm.dn[j];
              }
              int qf = qs + m * qt;
              if (bnd) {
                dk_face[(c0 * 6 + 2 * a + side0) * m2 + qf] = W * (-gxm * rm + th * xm * grm);
              } else {
                double dummy[3], dsd;
                side_eval(&o, cp, a, 0, qs, qt, n, dummy, &dsd, &dp);
                double xp = 0, rp = 0, gxp = 0, grp = 0;
                for (int j = 0; j < P3; ++j) {
                  xp += x[cp * P3 + j] * dp.phi[j]; rp += r[cp * P3 + j] * dp.phi[j];
                  gxp += x[cp * P3 + j] * dp.dn[j]; grp += r[cp * P3 + j] * dp.dn[j];
                }
                double jx = xm - xp, jr = rm - rp;
                dk_face[(cm * 6 + 2 * a + 1) * m2 + qf] = W * 0.5 * (-gxm * jr + th * jx * grm);
                dk_face[(cp * 6 + 2 * a) * m2 + qf] = W * 0.5 * (-gxp * jr + th * jx * grp);
              }
            }
        }
  }
  return 0;
}

int64_t oracle_assemble_coo(const oracle_problem *pb, int64_t cap, int64_t *rows, int64_t *cols,
                            double *vals) {
  octx o;
  if (ctx_init(&o, pb)) return INT64_MIN;
  const int L = o.L;
  int64_t nface = 0;
  for (int a = 0; a < 3; ++a) {
    int t1, t2;
    tangential_axes(a, &t1, &t2);
    nface += (int64_t)(o.n[a] - 1) * o.n[t1] * o.n[t2];
  }
  int64_t nbf = 2 * ((int64_t)o.n[0] * o.n[1] + (int64_t)o.n[1] * o.n[2] + (int64_t)o.n[0] * o.n[2]);
  int64_t need = o.ncell * L * L + nface * 4 * L * L + nbf * L * L;
  if (need > cap) return -need;
  double *e = calloc((size_t)6 * L, sizeof(double));
  if (!e) return INT64_MIN;
  double *z = e + L, *ym = e + 2 * L, *yp = e + 3 * L;
  int64_t cnt = 0;
  /* local dof -> global index */
#define GIDX(c, i) (o.pb->problem == 0 ? (c) * o.P3 + (i) \
                    : ((i) < 3 * o.P3 ? (c) * 3 * o.P3 + (i) : o.ncell * 3 * o.P3 + (c) * o.PP3 + (i) - 3 * o.P3))
  for (int64_t c = 0; c < o.ncell; ++c)
    for (int j = 0; j < L; ++j) {
      memset(e, 0, sizeof(double) * L);
      e[j] = 1.0;
      memset(ym, 0, sizeof(double) * L);
      vol_local(&o, c, e, ym);
      for (int i = 0; i < L; ++i) { rows[cnt] = GIDX(c, i); cols[cnt] = GIDX(c, j); vals[cnt++] = ym[i]; }
    }
  for (int a = 0; a < 3; ++a) {
    int t1, t2;
    tangential_axes(a, &t1, &t2);
    for (int i2 = 0; i2 < o.n[t2]; ++i2)
      for (int i1 = 0; i1 < o.n[t1]; ++i1)
        for (int f = 0; f <= o.n[a]; ++f) {
          int64_t cm, cp;
          face_cells(&o, a, f, i1, i2, &cm, &cp);
          if (cm >= 0 && cp >= 0) {
            for (int s = 0; s < 2; ++s)
              for (int j = 0; j < L; ++j) {
                memset(e, 0, sizeof(double) * L);
                memset(z, 0, sizeof(double) * L);
                (s == 0 ? e : z)[j] = 1.0;
                memset(ym, 0, sizeof(double) * L);
                memset(yp, 0, sizeof(double) * L);
                face_local(&o, a, cm, 1, cp, e, z, ym, yp, 0);
                int64_t cj = s == 0 ? cm : cp;
                for (int i = 0; i < L; ++i) {
                  rows[cnt] = GIDX(cm, i); cols[cnt] = GIDX(cj, j); vals[cnt++] = ym[i];
                  rows[cnt] = GIDX(cp, i); cols[cnt] = GIDX(cj, j); vals[cnt++] = yp[i];
                }
              }
          } else {
            int64_t cb = cm >= 0 ? cm : cp;
            int side = cm >= 0 ? 1 : 0;
            if (!((pb->dirichlet_mask >> (2 * a + side)) & 1)) continue;
            for (int j = 0; j < L; ++j) {
              memset(e, 0, sizeof(double) * L);
              e[j] = 1.0;
              memset(ym, 0, sizeof(double) * L);
              face_local(&o, a, cb, side, -1, e, NULL, ym, NULL, 0);
              for (int i = 0; i < L; ++i) { rows[cnt] = GIDX(cb, i); cols[cnt] = GIDX(cb, j); vals[cnt++] = ym[i]; }
            }
          }
        }
  }
#undef GIDX
  free(e);
  return cnt;
}

int oracle_rhs(const oracle_problem *pb, const double *f_vol, const double *g_face, double *F) {
  octx o;
  if (ctx_init(&o, pb) || pb->problem != 0 || o.aniso) return 1;
  const int P3 = o.P3, m = o.m, m2 = m * m, m3 = m * m * m;
  static __thread side_data dm;
  double *phi = malloc(sizeof(double) * P3 * 4);
  if (!phi) return 2;
  double (*g)[3] = (double (*)[3])(phi + P3);
  memset(F, 0, sizeof(double) * o.ncell * P3);
  if (f_vol) {
    for (int64_t c = 0; c < o.ncell; ++c) {
      double V[8][3], J[3][3], Ji[3][3], xi[3];
      cell_vertices(&o, c, V);
      for (int q2 = 0; q2 < m; ++q2)
        for (int q1 = 0; q1 < m; ++q1)
          for (int q0 = 0; q0 < m; ++q0) {
            xi[0] = o.s[q0]; xi[1] = o.s[q1]; xi[2] = o.s[q2];
            map_jacobian(V, xi, J);
            double dJ = det3(J);
            inv3(J, dJ, Ji);
            basis3d(o.p, o.zv, xi, Ji, phi, g);
            double w = o.w[q0] * o.w[q1] * o.w[q2] * dJ * f_vol[c * m3 + q0 + m * (q1 + m * q2)];
            for (int i = 0; i < P3; ++i) F[c * P3 + i] += w * phi[i];
          }
    }
  }
  free(phi);
  if (g_face) {
    for (int a = 0; a < 3; ++a) {
      int t1, t2;
      tangential_axes(a, &t1, &t2);
      for (int i2 = 0; i2 < o.n[t2]; ++i2)
        for (int i1 = 0; i1 < o.n[t1]; ++i1)
          for (int side = 0; side < 2; ++side) {
            int cc[3];
            cc[t1] = i1; cc[t2] = i2; cc[a] = side ? o.n[a] - 1 : 0;
            if (!((pb->dirichlet_mask >> (2 * a + side)) & 1)) continue;
            int64_t c = cell_index(&o, cc);
            int lf = 2 * a + side;
            double gam = penalty(&o, a, c, side, -1);
            for (int qt = 0; qt < m; ++qt)
              for (int qs = 0; qs < m; ++qs) {
                double n[3], ds;
                side_eval(&o, c, a, side, qs, qt, NULL, n, &ds, &dm);
                double W = o.w[qs] * o.w[qt] * ds;
                double gv = g_face[(c * 6 + lf) * m2 + qs + m * qt];
                double kap = kappa_face_at(&o, c, lf, qs, qt);
                for (int i = 0; i < P3; ++i)
                  F[c * P3 + i] += W * gv * (pb->theta * kap * dm.dn[i] + gam * dm.phi[i]);
              }
          }
    }
  }
  return 0;
}

/* Semilinear reaction (the nonlinear Jacobian action of Sec. 3's discussion, with a cubic
 * reaction chosen here): residual operator r(u)(v) = a(u, v) + beta (u^3, v), and its
 * Jacobian action at a linearisation point u0, J(u0) w = A w + 3 beta (u0^2 w, v).
 * mode 0: y = A w + beta (w^3, v) (u0 unused); mode 1: y = A w + 3 beta (u0^2 w, v).
 * The reaction integrals use the operator's Gauss rule and full basis evaluation. */
int oracle_semilinear(const oracle_problem *pb, double beta, int mode, const double *u0, const double *w,
                      double *y) {
  if (pb->problem != 0 || (mode != 0 && mode != 1) || (mode == 1 && !u0)) return 1;
  int st = oracle_apply(pb, 0, w, y);
  if (st) return st;
  octx o;
  if (ctx_init(&o, pb) || o.aniso) return 1;
  const int P3 = o.P3, m = o.m, L = o.L;
  double *we = malloc(sizeof(double) * 3 * L);
  if (!we) return 2;
  double *ue = we + L, *ye = we + 2 * L;
  static __thread double phi[OMAXP3], g[OMAXP3][3];
  for (int64_t c = 0; c < o.ncell; ++c) {
    double V[8][3], J[3][3], Ji[3][3], xi[3];
    gather(&o, c, w, we);
    if (mode == 1) gather(&o, c, u0, ue);
    memset(ye, 0, sizeof(double) * L);
    cell_vertices(&o, c, V);
    for (int q2 = 0; q2 < m; ++q2)
      for (int q1 = 0; q1 < m; ++q1)
        for (int q0 = 0; q0 < m; ++q0) {
          xi[0] = o.s[q0]; xi[1] = o.s[q1]; xi[2] = o.s[q2];
          const double W = o.w[q0] * o.w[q1] * o.w[q2];
          map_jacobian(V, xi, J);
          const double dJ = det3(J);
          inv3(J, dJ, Ji);
          basis3d(o.p, o.zv, xi, Ji, phi, g);
          double wq = 0.0, uq = 0.0;
          for (int j = 0; j < P3; ++j) {
            wq += we[j] * phi[j];
            if (mode == 1) uq += ue[j] * phi[j];
          }
          const double coef = mode == 0 ? beta * wq * wq * wq : 3.0 * beta * uq * uq * wq;
          for (int i = 0; i < P3; ++i) ye[i] += W * dJ * coef * phi[i];
        }
    scatter_add(&o, c, ye, y);
  }
  free(we);
  return 0;
}
