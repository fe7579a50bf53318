// Reference-element tables of the CUDA path (host, long double, rounded once).
//
// Quadrature (Sec. 2.1, "tensor product of 1D quadrature rules"): Gauss-Legendre nodes
// are the eigenvalues of the symmetric tridiagonal Jacobi matrix of the Legendre
// recurrence, found by Sturm-sequence bisection; weights from the Christoffel function
// w_i = 1 / sum_j (j + 1/2) P_j(t_i)^2. The local basis (left open by Sec. 2.1) is the
// Lagrange basis on the Gauss-Lobatto-Legendre points: 0, 1 and the roots of P_k',
// which are the eigenvalues of the Jacobi matrix of the Jacobi(1,1) recurrence.
//
// The kernels never evaluate the GLL basis at faces: they first interpolate a cell's
// coefficients to the Gauss points (matrix `interp`, Eq. lowcomplex with A^(i)), then
// use the Lagrange basis on the Gauss points themselves, whose derivative at the
// points is the m x m matrix `dcol` and whose traces at xi = 0, 1 are e0/e1 (d0/d1 for
// the derivative). This is exact whenever m >= k+1.
#include <math.h>
#include <string.h>

#include "dg_internal.h"

typedef long double ld;

// Number of eigenvalues < x of the symmetric tridiagonal matrix (zero diagonal,
// off-diagonal b[0..n-2]).
static int sturm_count(int n, const ld *b, ld x) {
  int cnt = 0;
  ld d = -x;
  if (d < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    ld prev = (d == 0) ? 1e-300L : d;
    d = -x - b[i - 1] * b[i - 1] / prev;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// All eigenvalues (ascending) by bisection on [-1, 1].
static void tridiag_eigs(int n, const ld *b, ld *ev) {
  for (int i = 0; i < n; ++i) {
    ld lo = -1.0L, hi = 1.0L;
    for (int it = 0; it < 200; ++it) {
      ld mid = 0.5L * (lo + hi);
      if (sturm_count(n, b, mid) > i) hi = mid; else lo = mid;
      if (hi - lo < 1e-30L) break;
    }
    ev[i] = 0.5L * (lo + hi);
  }
}

static void gauss_legendre(int m, ld *t, ld *w) {
  ld b[DG_MAXM];
  for (int i = 0; i + 1 < m; ++i) {
    ld j = i + 1;
    b[i] = j / sqrtl(4.0L * j * j - 1.0L);
  }
  tridiag_eigs(m, b, t);
  for (int i = 0; i < m; ++i) {
    ld p0 = 1.0L, p1 = t[i], s = 0.5L;  // (j + 1/2) P_j^2 for j = 0
    if (m > 1) s += 1.5L * p1 * p1;
    for (int j = 2; j < m; ++j) {
      ld p2 = ((2.0L * j - 1.0L) * t[i] * p1 - (j - 1.0L) * p0) / j;
      p0 = p1;
      p1 = p2;
      s += (j + 0.5L) * p2 * p2;
    }
    w[i] = 1.0L / s;
  }
}

static void gll_points(int k, ld *z) {
  // on [-1,1]: -1, roots of P_k' (Jacobi(1,1) degree k-1), +1
  z[0] = -1.0L;
  z[k] = 1.0L;
  if (k >= 2) {
    ld b[DG_MAXP], ev[DG_MAXP];
    for (int n = 1; n <= k - 2; ++n) b[n - 1] = sqrtl((ld)n * (n + 2) / ((2.0L * n + 1) * (2.0L * n + 3)));
    tridiag_eigs(k - 1, b, ev);
    for (int i = 0; i < k - 1; ++i) z[i + 1] = ev[i];
  }
}

// Barycentric weights lambda_j = 1 / prod_{i != j} (z_j - z_i).
static void bary_weights(int n, const ld *z, ld *lam) {
  for (int j = 0; j < n; ++j) {
    ld p = 1.0L;
    for (int i = 0; i < n; ++i)
      if (i != j) p *= (z[j] - z[i]);
    lam[j] = 1.0L / p;
  }
}

// Values and derivatives of all Lagrange polynomials on z at point t.
static void lagrange_at(int n, const ld *z, const ld *lam, ld t, ld *val, ld *der) {
  int hit = -1;
  for (int i = 0; i < n; ++i)
    if (t == z[i]) hit = i;
  if (hit >= 0) {
    for (int r = 0; r < n; ++r) {
      val[r] = (r == hit) ? 1.0L : 0.0L;
      if (r == hit) {
        ld s = 0.0L;
        for (int i = 0; i < n; ++i)
          if (i != hit) s += 1.0L / (z[hit] - z[i]);
        der[r] = s;
      } else {
        der[r] = (lam[r] / lam[hit]) / (z[hit] - z[r]);
      }
    }
    return;
  }
  ld node = 1.0L;
  for (int i = 0; i < n; ++i) node *= (t - z[i]);
  for (int j = 0; j < n; ++j) {
    val[j] = node * lam[j] / (t - z[j]);
    ld s = 0.0L;
    for (int i = 0; i < n; ++i)
      if (i != j) s += 1.0L / (t - z[i]);
    der[j] = val[j] * s;
  }
}

int dg_build_tables(int k, int m, bool with_pressure, HostTables *T) {
  if (k < 1 || k + 1 > DG_MAXP || m < k + 1 || m > DG_MAXM) return 1;
  memset(T, 0, sizeof(*T));
  T->k = k;
  T->p = k + 1;
  T->m = m;
  ld t[DG_MAXM], w[DG_MAXM], s[DG_MAXM];
  gauss_legendre(m, t, w);
  for (int q = 0; q < m; ++q) {
    s[q] = (1.0L + t[q]) / 2.0L;
    T->gauss_s[q] = (double)s[q];
    T->gauss_w[q] = (double)(w[q] / 2.0L);
  }
  ld z[DG_MAXP], zl[DG_MAXP], lam[DG_MAXP], val[DG_MAXP], der[DG_MAXP];
  gll_points(k, zl);
  for (int j = 0; j <= k; ++j) {
    z[j] = (1.0L + zl[j]) / 2.0L;
    T->gll[j] = (double)z[j];
  }
  bary_weights(k + 1, z, lam);
  for (int q = 0; q < m; ++q) {
    lagrange_at(k + 1, z, lam, s[q], val, der);
    for (int j = 0; j <= k; ++j) T->interp[q * T->p + j] = (double)val[j];
  }
  lagrange_at(k + 1, z, lam, 0.0L, val, der);
  for (int j = 0; j <= k; ++j) T->gd0[j] = (double)der[j];
  lagrange_at(k + 1, z, lam, 1.0L, val, der);
  for (int j = 0; j <= k; ++j) T->gd1[j] = (double)der[j];
  ld lg[DG_MAXM], vg[DG_MAXM], dg[DG_MAXM];
  bary_weights(m, s, lg);
  for (int q = 0; q < m; ++q) {
    lagrange_at(m, s, lg, s[q], vg, dg);
    for (int r = 0; r < m; ++r) T->dcol[q * m + r] = (double)dg[r];
  }
  lagrange_at(m, s, lg, 0.0L, vg, dg);
  for (int r = 0; r < m; ++r) { T->e0[r] = (double)vg[r]; T->d0[r] = (double)dg[r]; }
  lagrange_at(m, s, lg, 1.0L, vg, dg);
  for (int r = 0; r < m; ++r) { T->e1[r] = (double)vg[r]; T->d1[r] = (double)dg[r]; }
  if (with_pressure) {
    if (k < 2) return 1;
    T->pp = k;
    ld zp[DG_MAXP], lp[DG_MAXP];
    gll_points(k - 1, zl);
    for (int j = 0; j < k; ++j) zp[j] = (1.0L + zl[j]) / 2.0L;
    bary_weights(k, zp, lp);
    for (int q = 0; q < m; ++q) {
      lagrange_at(k, zp, lp, s[q], val, der);
      for (int j = 0; j < k; ++j) T->interp_p[q * k + j] = (double)val[j];
    }
  }
  return 0;
}
