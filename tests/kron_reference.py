"""Independent construction of the affine SIPG-DG matrices from 1D factors.

On an axis-aligned Cartesian mesh the bilinear forms of Eq. (diffreac_weak) (Sec. 5.2)
and Eq. (stokes_weak) (Sec. 5.3) with constant coefficients separate into Kronecker
products of 1D matrices: each x-face term is a 1D point term in x times the 1D mass
matrices in y and z, and each volume term is a 1D stiffness/mass product. The 1D
matrices are built here by exact polynomial integration with numpy, on GLL nodes
taken as the roots of P_k' from numpy; nothing is shared with the oracle. A test that
compares the oracle's assembled matrix with this one pins every sign, factor and
index convention of the affine operator.
"""
from __future__ import annotations

import numpy as np
import numpy.polynomial.legendre as npleg
import numpy.polynomial.polynomial as npp
import scipy.sparse as sp


def gll_points(k: int) -> np.ndarray:
    """GLL points on [0,1]: 0, 1 and the roots of P_k' (numpy's Legendre class)."""
    if k == 1:
        t = np.array([-1.0, 1.0])
    else:
        inner = np.sort(np.real(npleg.Legendre.basis(k).deriv().roots()))
        t = np.concatenate([[-1.0], inner, [1.0]])
    return (t + 1.0) / 2.0


def lagrange_polys(z: np.ndarray):
    """Power-series coefficients of the Lagrange polynomials on nodes z."""
    out = []
    for j in range(len(z)):
        c = np.array([1.0])
        for i in range(len(z)):
            if i != j:
                c = npp.polymul(c, np.array([-z[i], 1.0]) / (z[j] - z[i]))
        out.append(c)
    return out


def _int01(c) -> float:
    ci = npp.polyint(c)
    return float(npp.polyval(1.0, ci) - npp.polyval(0.0, ci))


class Basis1D:
    """Lagrange basis on nodes z: values/derivatives by the product formula, integrals
    of products by a 24-point numpy Gauss rule (exact up to degree 47)."""

    def __init__(self, z: np.ndarray):
        self.z = np.asarray(z, dtype=np.float64)
        self.n = len(z)
        self.P = lagrange_polys(z)  # power series, only for low-degree moments in tests
        t, w = npleg.leggauss(24)
        self._qs, self._qw = (t + 1) / 2, w / 2
        self._V = np.array([[self.val(j, s) for j in range(self.n)] for s in self._qs])
        self._D = np.array([[self.der(j, s) for j in range(self.n)] for s in self._qs])

    def val(self, j, t):
        z = self.z
        return float(np.prod([(t - z[i]) / (z[j] - z[i]) for i in range(self.n) if i != j]))

    def der(self, j, t):
        z = self.z
        tot = 0.0
        for l in range(self.n):
            if l == j:
                continue
            term = 1.0 / (z[j] - z[l])
            for i in range(self.n):
                if i != j and i != l:
                    term *= (t - z[i]) / (z[j] - z[i])
            tot += term
        return tot

    def table(self, kind):
        return self._V if kind == "v" else self._D


def _gram(bi: "Basis1D", ki: str, bj: "Basis1D", kj: str) -> np.ndarray:
    """int_0^1 f_i g_j for f, g basis values ('v') or derivatives ('d')."""
    return (bi.table(ki) * bi._qw[:, None]).T @ bj.table(kj)


def mass_1d(bi: Basis1D, bj: Basis1D, n: int, h: float):
    """Block-diagonal 1D mass matrix h*int l_i l_j over n cells (rows bi, cols bj)."""
    loc = _gram(bi, "v", bj, "v")
    return sp.kron(sp.identity(n), h * loc).tocsr()


def sipg_1d(b: Basis1D, n: int, h: float, gamma: float, theta: float, bc_lo: bool, bc_hi: bool):
    """1D SIPG matrix for -u'' on n uniform cells of size h: volume stiffness plus point
    terms -{u'}[v] + theta [u]{v'} + gamma [u][v] at interior points and, where a
    boundary is Dirichlet, the same with jump = average = trace and the outward normal."""
    p = b.n
    N = n * p
    A = np.zeros((N, N))
    stiff = _gram(b, "d", b, "d") / h
    for e in range(n):
        A[e * p:(e + 1) * p, e * p:(e + 1) * p] += stiff

    def trace(e, t):
        """(global index, value, physical derivative) of the basis of cell e at local t."""
        return [(e * p + j, b.val(j, t), b.der(j, t) / h) for j in range(p)]

    def add_point(sides):
        # sides: list of (trace list, sign in jump, weight in average); normal +x
        for (tr_u, su, wu) in sides:
            for (gu, vu, du) in tr_u:
                for (tr_v, sv, wv) in sides:
                    for (gv, vv, dv) in tr_v:
                        A[gv, gu] += (-(wu * du) * (sv * vv) + theta * (su * vu) * (wv * dv)
                                      + gamma * (su * vu) * (sv * vv))

    for e in range(n - 1):
        add_point([(trace(e, 1.0), 1.0, 0.5), (trace(e + 1, 0.0), -1.0, 0.5)])
    # boundary: with outward normal nrm, n.grad u = nrm * u'; write as jump sign = 1 and
    # fold the normal into the derivative weight (flux and symmetry terms both carry n)
    if bc_lo:
        add_point([(trace(0, 0.0), 1.0, -1.0)])
    if bc_hi:
        add_point([(trace(n - 1, 1.0), 1.0, 1.0)])
    return sp.csr_matrix(A)


def div_1d(bq: Basis1D, bu: Basis1D, n: int, bc_lo: bool, bc_hi: bool):
    """1D factor of b(u, q) = -(u', q) + ([u] n, {q}) (rows q, cols u), unscaled by h
    (the derivative's 1/h cancels the length element h)."""
    pq, pu = bq.n, bu.n
    B = np.zeros((n * pq, n * pu))
    loc = _gram(bq, "v", bu, "d")
    for e in range(n):
        B[e * pq:(e + 1) * pq, e * pu:(e + 1) * pu] -= loc
    for e in range(n - 1):
        for (eu, tu, su) in ((e, 1.0, 1.0), (e + 1, 0.0, -1.0)):
            for j in range(pu):
                ju = su * bu.val(j, tu)
                for (eq, tq) in ((e, 1.0), (e + 1, 0.0)):
                    for l in range(pq):
                        B[eq * pq + l, eu * pu + j] += ju * 0.5 * bq.val(l, tq)
    if bc_lo:
        for j in range(pu):
            for l in range(pq):
                B[l, j] += bu.val(j, 0.0) * (-1.0) * bq.val(l, 0.0)
    if bc_hi:
        e = n - 1
        for j in range(pu):
            for l in range(pq):
                B[e * pq + l, e * pu + j] += bu.val(j, 1.0) * 1.0 * bq.val(l, 1.0)
    return sp.csr_matrix(B)


def _perm(nx, ny, nz, p):
    """Kronecker index (ix fastest over nx*p0, then iy, then iz) -> cell-major index; p is
    the number of basis points per direction, or a triple (p0, p1, p2)."""
    p0, p1, p2 = (p, p, p) if np.isscalar(p) else p
    ix = np.arange(nx * p0)
    iy = np.arange(ny * p1)
    iz = np.arange(nz * p2)
    IZ, IY, IX = np.meshgrid(iz, iy, ix, indexing="ij")
    cx, j0 = IX // p0, IX % p0
    cy, j1 = IY // p1, IY % p1
    cz, j2 = IZ // p2, IZ % p2
    g = (cx + nx * (cy + ny * cz)) * (p0 * p1 * p2) + j0 + p0 * (j1 + p1 * j2)
    return g.ravel()


def _reorder(K, rperm, cperm, nrow, ncol):
    K = K.tocoo()
    return sp.csr_matrix((K.data, (rperm[K.row], cperm[K.col])), shape=(nrow, ncol))


def gamma_axis(k, n_a, alpha, pen_mode):
    return alpha * k * (k + 1) * n_a if pen_mode == 0 else alpha * k * (k + 2) * n_a


def scalar_matrix(nx, ny, nz, k, c=1.0, theta=-1.0, alpha=2.0, pen_mode=0, mask=0b111111, kappa=1.0,
                  degrees=None):
    """Affine unit-cube SIPG matrix (constant kappa) in the cell-major DOF order; degrees
    (k_0, k_1, k_2) gives each direction its own basis and the face penalty the degree along
    the face normal."""
    ks = tuple(degrees) if degrees is not None else (k, k, k)
    bs = [Basis1D(gll_points(ka)) for ka in ks]
    n = (nx, ny, nz)
    M = [mass_1d(bs[a], bs[a], n[a], 1.0 / n[a]) for a in range(3)]
    S = [sipg_1d(bs[a], n[a], 1.0 / n[a], gamma_axis(ks[a], n[a], alpha, pen_mode) / kappa, theta,
                 bool(mask >> (2 * a) & 1), bool(mask >> (2 * a + 1) & 1)) for a in range(3)]
    K = (kappa * (sp.kron(M[2], sp.kron(M[1], S[0])) + sp.kron(M[2], sp.kron(S[1], M[0]))
                  + sp.kron(S[2], sp.kron(M[1], M[0])))
         + c * sp.kron(M[2], sp.kron(M[1], M[0])))
    perm = _perm(nx, ny, nz, tuple(ka + 1 for ka in ks))
    N = K.shape[0]
    return _reorder(K, perm, perm, N, N)


def stokes_matrix(nx, ny, nz, k, mu=1.0, theta=-1.0, alpha=2.0, pen_mode=0, mask=0b111101):
    """Affine unit-cube DG Stokes block matrix [[A_v, B^T], [B, 0]] in the layout
    [u: ncell x 3 x (k+1)^3 | p: ncell x k^3]."""
    bv = Basis1D(gll_points(k))
    bp = Basis1D(gll_points(k - 1))
    n = (nx, ny, nz)
    ncell = nx * ny * nz
    p, pp = k + 1, k
    P3, PP3 = p ** 3, pp ** 3
    Av = scalar_matrix(nx, ny, nz, k, c=0.0, theta=theta, alpha=alpha, pen_mode=pen_mode, mask=mask, kappa=mu)
    Mvv = [mass_1d(bv, bv, n[a], 1.0 / n[a]) for a in range(3)]
    Mpv = [mass_1d(bp, bv, n[a], 1.0 / n[a]) for a in range(3)]
    Dpv = [div_1d(bp, bv, n[a], bool(mask >> (2 * a) & 1), bool(mask >> (2 * a + 1) & 1)) for a in range(3)]
    # B_c: -(d_c u_c, q) + ([u_c] n_c, {q}) = Dpv in direction c times mixed masses elsewhere
    # with the physical scaling h_b h_c (the derivative direction's h cancels)
    perm_v = _perm(nx, ny, nz, p)
    perm_p = _perm(nx, ny, nz, pp)
    N = ncell * (3 * P3 + PP3)
    rows, cols, vals = [], [], []
    Av = Av.tocoo()
    cell_v = Av.row // P3
    cell_vc = Av.col // P3
    for comp in range(3):
        r = (cell_v * 3 + comp) * P3 + Av.row % P3
        cc = (cell_vc * 3 + comp) * P3 + Av.col % P3
        rows.append(r); cols.append(cc); vals.append(Av.data)
    for comp in range(3):
        fac = [Mpv[a] for a in range(3)]
        fac[comp] = Dpv[comp]
        Bc = sp.kron(fac[2], sp.kron(fac[1], fac[0])).tocoo()
        qi = perm_p[Bc.row]
        ui = perm_v[Bc.col]
        rq = ncell * 3 * P3 + qi
        cu = (ui // P3 * 3 + comp) * P3 + ui % P3
        rows += [rq, cu]; cols += [cu, rq]; vals += [Bc.data, Bc.data]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
