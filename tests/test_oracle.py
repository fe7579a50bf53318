"""Pins for the CPU oracle against facts that do not come from the oracle itself:
library quadrature rules, closed forms, an independent Kronecker construction of the
affine operator, exactness identities, the paper's manufactured solutions (Sec. 5.2,
Sec. 5.3), convergence rates and finite differences."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest
import scipy.sparse.linalg as spla

import kron_reference as kr
import oracle
from paper_1812_08075_gb300 import workloads as wl


# ---------------------------------------------------------------- 1D rules (Sec. 2.1)

@pytest.mark.parametrize("m", range(1, 9))
def test_gauss_rule_matches_numpy_and_is_exact(m):
    s, w = oracle.gauss_rule(m)
    t, wt = npleg.leggauss(m)
    np.testing.assert_allclose(s, (t + 1) / 2, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, wt / 2, rtol=0, atol=1e-15)  # numpy is ~4e-16 off at m=8
    for d in range(2 * m):  # exact up to degree 2m-1
        assert abs(np.sum(w * s ** d) - 1.0 / (d + 1)) < 5e-16
    assert abs(np.sum(w * s ** (2 * m)) - 1.0 / (2 * m + 1)) > 1e-12  # degree 2m is not


def test_gll_nodes_closed_forms_and_numpy_roots():
    np.testing.assert_allclose(oracle.gll_nodes(1), [0, 1], atol=0)
    np.testing.assert_allclose(oracle.gll_nodes(2), [0, 0.5, 1], atol=1e-16)
    r5 = 1 / np.sqrt(5)
    np.testing.assert_allclose(oracle.gll_nodes(3), [0, (1 - r5) / 2, (1 + r5) / 2, 1], atol=1e-16)
    r37 = np.sqrt(3 / 7)
    np.testing.assert_allclose(oracle.gll_nodes(4), [0, (1 - r37) / 2, 0.5, (1 + r37) / 2, 1], atol=1e-16)
    for k in range(1, 8):
        np.testing.assert_allclose(oracle.gll_nodes(k), kr.gll_points(k), atol=1e-14)


# ------------------------------------------- affine operator vs independent construction

@pytest.mark.parametrize("n,k,theta,c,pen_mode,mask", [
    ((3, 2, 4), 2, -1.0, 1.0, 0, 0b111111),
    ((2, 3, 2), 1, 1.0, 0.5, 1, 0b101101),
    ((2, 2, 2), 3, 0.0, 2.0, 0, 0b111111),
    ((1, 2, 3), 2, -1.0, 0.0, 1, 0b010110),
    ((2, 2, 2), 4, -1.0, 1.0, 0, 0b011011),
    ((2, 1, 1), 5, -1.0, 1.0, 0, 0b111111),
])
def test_affine_scalar_matches_kronecker(n, k, theta, c, pen_mode, mask):
    p = oracle.Problem(*n, k, c=c, theta=theta, pen_mode=pen_mode, dirichlet_mask=mask)
    A = p.assemble()
    K = kr.scalar_matrix(*n, k, c=c, theta=theta, pen_mode=pen_mode, mask=mask)
    assert abs(A - K).max() <= 1e-11 * abs(K).max()


def test_affine_scalar_overintegration_equals_exact():
    # affine integrands are polynomials: m = k+1 is already exact, m = k+3 must agree
    p1 = oracle.Problem(2, 3, 2, 2)
    p2 = oracle.Problem(2, 3, 2, 2, m=5)
    A1, A2 = p1.assemble(), p2.assemble()
    assert abs(A1 - A2).max() <= 1e-13 * abs(A1).max()


@pytest.mark.parametrize("n,k,mask", [((2, 2, 2), 2, 0b111101), ((3, 2, 2), 3, 0b111101), ((2, 2, 1), 2, 0b111111)])
def test_affine_stokes_matches_kronecker(n, k, mask):
    p = oracle.Problem(*n, k, problem="stokes", dirichlet_mask=mask)
    A = p.assemble()
    K = kr.stokes_matrix(*n, k, mask=mask)
    assert abs(A - K).max() <= 1e-12 * abs(K).max()


# ------------------------------------------------------------ matrix-free vs assembled

def _trilinear_problem(n=(3, 2, 2), k=2, seed=1, **kw):
    v = wl.perturbed_vertices(*n, seed=seed)
    return oracle.Problem(*n, k, vertices=v, **kw)


def test_apply_equals_assembled_and_transpose():
    p = _trilinear_problem(theta=1.0)  # NIPG: A is not symmetric
    km, kf = wl.lognormal_kappa(p.ncell, p.m, seed=2)
    p.kappa_vol, p.kappa_face = km, kf
    A = p.assemble()
    x = wl.uniform_vector(p.ndofs(), 0)
    y = p.apply(x)
    yt = p.apply(x, transpose=True)
    np.testing.assert_allclose(y, A @ x, rtol=0, atol=1e-13 * abs(y).max())
    np.testing.assert_allclose(yt, A.T @ x, rtol=0, atol=1e-13 * abs(yt).max())
    assert abs(A - A.T).max() > 1e-3 * abs(A).max()


@pytest.mark.parametrize("problem", ["scalar", "stokes"])
def test_apply_cells_gather_equals_apply(problem):
    p = _trilinear_problem(n=(3, 3, 2), k=2, problem=problem,
                           dirichlet_mask=0b111101 if problem == "stokes" else 0b111111)
    if problem == "scalar":
        p.kappa_vol, p.kappa_face = wl.lognormal_kappa(p.ncell, p.m, seed=2)
    x = wl.uniform_vector(p.ndofs(), 0)
    y = p.apply(x)
    cells = np.arange(p.ncell)
    yc = p.apply_cells(x, cells, nthreads=3)
    if problem == "scalar":
        np.testing.assert_allclose(yc.ravel(), y, rtol=0, atol=1e-13 * abs(y).max())
    else:
        P3, PP3 = 27, 8
        yu = y[: p.ncell * 3 * P3].reshape(p.ncell, 3 * P3)
        yp = y[p.ncell * 3 * P3:].reshape(p.ncell, PP3)
        np.testing.assert_allclose(yc[:, :3 * P3], yu, rtol=0, atol=1e-13 * abs(y).max())
        np.testing.assert_allclose(yc[:, 3 * P3:], yp, rtol=0, atol=1e-13 * abs(y).max())


# ---------------------------------------------------------- trilinear geometry pins

def test_trilinear_symmetry_with_pointwise_kappa():
    p = _trilinear_problem(n=(2, 3, 2), k=2)
    p.kappa_vol, p.kappa_face = wl.lognormal_kappa(p.ncell, p.m, seed=2)
    A = p.assemble()
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mass_closed_form_on_perturbed_mesh(k):
    # kappa = 0 and alpha = 0 leave c*M; 1^T M 1 = |Omega| = 1 exactly (detJ is a
    # polynomial of degree <= 2 per direction, integrated exactly by m = k+1 >= 2)
    n = (3, 2, 3)
    p = _trilinear_problem(n=n, k=k, c=1.7, pen_alpha=0.0)
    p.kappa_vol = np.zeros(p.ncell * p.m ** 3)
    p.kappa_face = np.zeros(p.ncell * 6 * p.m ** 2)
    one = np.ones(p.ndofs())
    assert abs(one @ p.apply(one) - 1.7) < 1e-13


@pytest.mark.parametrize("k", [1, 2, 3])
def test_penalty_closed_form_on_perturbed_mesh(k):
    # x = 1: gradients vanish and interior jumps vanish, so 1^T A 1 = c|Omega| + sum over
    # the six planar boundary faces of gamma_F |F| with gamma_F = alpha k(k+1) n_a
    n = (3, 2, 4)
    alpha = 2.0
    p = _trilinear_problem(n=n, k=k, c=1.0, pen_alpha=alpha)
    p.kappa_vol, p.kappa_face = wl.lognormal_kappa(p.ncell, p.m, seed=2)
    one = np.ones(p.ndofs())
    expect = 1.0 + sum(2 * alpha * k * (k + 1) * n[a] for a in range(3))
    assert abs(one @ p.apply(one) - expect) < 1e-12 * expect


def _trilinear_point(V8, xi):
    """Physical point of reference point xi in the cell with corner vertices V8[8,3]."""
    x = np.zeros(3)
    for a in range(8):
        b = [(a >> d) & 1 for d in range(3)]
        w = np.prod([xi[d] if b[d] else 1 - xi[d] for d in range(3)])
        x += w * V8[a]
    return x


def _cell_corners(v, n, c):
    nx, ny, nz = n
    cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
    out = np.zeros((8, 3))
    for a in range(8):
        i, j, l = cx + (a & 1), cy + ((a >> 1) & 1), cz + ((a >> 2) & 1)
        out[a] = v[i + (nx + 1) * (j + (ny + 1) * l)]
    return out


def _interpolate(v, n, k, func, ncomp=1):
    """Nodal interpolant on GLL nodes (numpy-derived) mapped through each cell."""
    z = kr.gll_points(k)
    p = k + 1
    ncell = n[0] * n[1] * n[2]
    out = np.zeros((ncell, ncomp, p ** 3))
    for c in range(ncell):
        V8 = _cell_corners(v, n, c)
        for j2 in range(p):
            for j1 in range(p):
                for j0 in range(p):
                    x = _trilinear_point(V8, (z[j0], z[j1], z[j2]))
                    out[c, :, j0 + p * (j1 + p * j2)] = func(x)
    return out


def _interior_cells(n):
    nx, ny, nz = n
    c = np.arange(nx * ny * nz)
    cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
    return c[(cx > 0) & (cx < nx - 1) & (cy > 0) & (cy < ny - 1) & (cz > 0) & (cz < nz - 1)]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_solution_consistency_on_perturbed_mesh(k):
    # u linear in x is exactly representable on trilinear cells; with kappa = 1, c = 0,
    # -div grad u = 0 and every volume/face integrand touching a cell away from the
    # boundary is a polynomial integrated exactly, so (A u_I) vanishes there.
    n = (4, 3, 3)
    v = wl.perturbed_vertices(*n, seed=1)
    p = oracle.Problem(*n, k, vertices=v, c=0.0)
    u = _interpolate(v, n, k, lambda x: 0.3 + 1.1 * x[0] - 0.7 * x[1] + 0.4 * x[2])[:, 0, :]
    y = p.apply(u.ravel()).reshape(p.ncell, -1)
    inner = _interior_cells(n)
    assert inner.size > 0
    assert abs(y[inner]).max() < 1e-13 * abs(y).max()
    assert abs(y).max() > 1e-3  # boundary cells see the boundary terms


def test_paper_manufactured_solution_affine():
    # Sec. 5.2: g = |x|^2 solves -div grad u + c u = f with kappa = 1 (our scalar reading),
    # c = 1, f = -6 + |x|^2. On affine cells every integrand is polynomial, so for cells
    # away from the boundary A g_I = (f, phi_i) exactly.
    n, k = (4, 3, 3), 2
    v = wl.unit_cube_vertices(*n)
    p = oracle.Problem(*n, k, c=1.0)
    u = _interpolate(v, n, k, lambda x: float(x @ x))[:, 0, :]
    y = p.apply(u.ravel()).reshape(p.ncell, -1)
    b = kr.Basis1D(kr.gll_points(k))
    import numpy.polynomial.polynomial as npp

    def mom(lo, h, j, power):
        # int_{lo}^{lo+h} x^power l_j((x-lo)/h) dx = h int_0^1 (lo + h t)^power l_j(t) dt
        poly = npp.polypow(np.array([lo, h]), power)
        ci = npp.polyint(npp.polymul(poly, b.P[j]))
        return h * (npp.polyval(1.0, ci) - npp.polyval(0.0, ci))

    hx = [1.0 / n[a] for a in range(3)]
    pp = k + 1
    for c in _interior_cells(n):
        cc = (c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1]))
        lo = [cc[a] * hx[a] for a in range(3)]
        for j2 in range(pp):
            for j1 in range(pp):
                for j0 in range(pp):
                    js = (j0, j1, j2)
                    m0 = [mom(lo[a], hx[a], js[a], 0) for a in range(3)]
                    m2 = [mom(lo[a], hx[a], js[a], 2) for a in range(3)]
                    f = -6 * m0[0] * m0[1] * m0[2] + m2[0] * m0[1] * m0[2] + m0[0] * m2[1] * m0[2] + m0[0] * m0[1] * m2[2]
                    assert abs(y[c, j0 + pp * (j1 + pp * j2)] - f) < 1e-13


@pytest.mark.parametrize("k", [2, 3])
def test_paper_stokes_manufactured_solution_affine(k):
    # Sec. 5.3: u = (4 y (1-y), 0, 0), p = 8 (1 - x) solve the Stokes problem with f = 0;
    # away from the boundary the block residual vanishes exactly on affine cells.
    n = (4, 4, 3)
    v = wl.unit_cube_vertices(*n)
    p = oracle.Problem(*n, k, problem="stokes", dirichlet_mask=0b111101)
    u = _interpolate(v, n, k, lambda x: np.array([4 * x[1] * (1 - x[1]), 0.0, 0.0]), ncomp=3)
    pr = _interpolate(v, n, k - 1, lambda x: 8 * (1 - x[0]))[:, 0, :]
    y = p.apply(np.concatenate([u.ravel(), pr.ravel()]))
    P3 = (k + 1) ** 3
    yu = y[: p.ncell * 3 * P3].reshape(p.ncell, 3 * P3)
    yp = y[p.ncell * 3 * P3:].reshape(p.ncell, k ** 3)
    inner = _interior_cells(n)
    assert inner.size > 0
    assert abs(yu[inner]).max() < 1e-12 and abs(yp[inner]).max() < 1e-12
    assert abs(yu).max() > 1e-3


def test_stokes_constant_pressure_closed_form_on_perturbed_mesh():
    # u = 0, p = 1: each cell's -(1, div v) + sum_F ({1}, [v].n) collapses by the
    # divergence theorem to -int over its Neumann faces (x = 1) of phi_i n_x ds.
    n, k = (3, 2, 2), 2
    v = wl.perturbed_vertices(*n, seed=1)
    p = oracle.Problem(*n, k, vertices=v, problem="stokes", dirichlet_mask=0b111101)
    P3, PP3 = (k + 1) ** 3, k ** 3
    x = np.concatenate([np.zeros(p.ncell * 3 * P3), np.ones(p.ncell * PP3)])
    y = p.apply(x)
    yu = y[: p.ncell * 3 * P3].reshape(p.ncell, 3, P3)
    yp = y[p.ncell * 3 * P3:]
    b = kr.Basis1D(kr.gll_points(k))
    W = np.array([kr._int01(b.P[j]) for j in range(k + 1)])
    expect = np.zeros_like(yu)
    pp = k + 1
    for c in range(p.ncell):
        if c % n[0] == n[0] - 1:
            for j2 in range(pp):
                for j1 in range(pp):
                    expect[c, 0, k + pp * (j1 + pp * j2)] = -(1 / n[1]) * (1 / n[2]) * W[j1] * W[j2]
    assert abs(yu - expect).max() < 1e-13
    assert abs(yp).max() < 1e-13


def test_stokes_symmetric_indefinite_inertia():
    p = _trilinear_problem(n=(2, 2, 2), k=2, problem="stokes", dirichlet_mask=0b111101)
    A = p.assemble().toarray()
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    ev = np.linalg.eigvalsh(A)
    npres = p.ncell * p.k ** 3
    assert np.sum(ev < -1e-10) == npres
    assert np.sum(np.abs(ev) < 1e-10) == 0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sipg_coercive_on_perturbed_mesh(k):
    p = _trilinear_problem(n=(2, 2, 2), k=k, c=0.0)
    ev = np.linalg.eigvalsh(p.assemble().toarray())
    assert ev.min() > 0


# ------------------------------------------------------------------ convergence

def _load_and_error_tools(v, n, k, mq):
    """Test-side quadrature (numpy Gauss, mq points) on each trilinear cell:
    returns per-cell lists of (weights*detJ, physical points, basis values)."""
    t, wt = npleg.leggauss(mq)
    s, w = (t + 1) / 2, wt / 2
    b = kr.Basis1D(kr.gll_points(k))
    p = k + 1
    B1 = np.array([[b.val(j, si) for j in range(p)] for si in s])  # [mq, p]
    # phi[(q0,q1,q2), j0 + p(j1 + p j2)] = l_j0(s_q0) l_j1(s_q1) l_j2(s_q2)
    phi = np.einsum("aj,bk,cl->abclkj", B1, B1, B1).reshape(mq ** 3, p ** 3)
    Q = np.array([(s[q0], s[q1], s[q2], w[q0] * w[q1] * w[q2])
                  for q0 in range(mq) for q1 in range(mq) for q2 in range(mq)])
    ncell = n[0] * n[1] * n[2]
    out = []
    for c in range(ncell):
        V8 = _cell_corners(v, n, c)
        X = np.zeros((Q.shape[0], 3))
        dJ = np.zeros(Q.shape[0])
        for qi, (a0, a1, a2, wq) in enumerate(Q):
            xi = (a0, a1, a2)
            X[qi] = _trilinear_point(V8, xi)
            J = np.zeros((3, 3))
            for a in range(8):
                bb = [(a >> d) & 1 for d in range(3)]
                f = [xi[d] if bb[d] else 1 - xi[d] for d in range(3)]
                df = [1.0 if bb[d] else -1.0 for d in range(3)]
                J[:, 0] += df[0] * f[1] * f[2] * V8[a]
                J[:, 1] += f[0] * df[1] * f[2] * V8[a]
                J[:, 2] += f[0] * f[1] * df[2] * V8[a]
            dJ[qi] = np.linalg.det(J) * wq
        out.append((dJ, X))
    return out, phi


@pytest.mark.parametrize("k,sizes,geom", [(1, (2, 4, 8), "affine"), (2, (2, 4, 8), "perturbed"), (3, (2, 4), "perturbed")])
def test_convergence_order(k, sizes, geom):
    # -div grad u + u = (3 pi^2 + 1) u, u = sin(pi x) sin(pi y) sin(pi z), u = 0 on the boundary
    errs = []
    for N in sizes:
        n = (N, N, N)
        v = wl.perturbed_vertices(*n, seed=1) if geom == "perturbed" else wl.unit_cube_vertices(*n)
        p = oracle.Problem(*n, k, vertices=v, c=1.0, pen_alpha=2.0)
        A = p.assemble()
        tools, phi = _load_and_error_tools(v, n, k, k + 3)
        F = np.zeros((p.ncell, (k + 1) ** 3))
        uex = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        for c, (wdJ, X) in enumerate(tools):
            F[c] = phi.T @ (wdJ * (3 * np.pi ** 2 + 1) * uex(X))
        uh = spla.spsolve(A.tocsc(), F.ravel()).reshape(p.ncell, -1)
        e2 = 0.0
        for c, (wdJ, X) in enumerate(tools):
            e2 += np.sum(wdJ * (phi @ uh[c] - uex(X)) ** 2)
        errs.append(np.sqrt(e2))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - (k + 1)) < 0.4, (errs, rates)


# --------------------------------------------------------------------- adjoint / dkappa

def _loss(p, x, b):
    r = p.apply(x) - b
    return 0.5 * float(r @ r)


def test_dkappa_matches_central_differences():
    p = _trilinear_problem(n=(2, 2, 3), k=2, theta=-1.0)
    kv, kf = wl.lognormal_kappa(p.ncell, p.m, seed=2)
    p.kappa_vol, p.kappa_face = kv, kf
    x = wl.uniform_vector(p.ndofs(), 3)
    b = wl.uniform_vector(p.ndofs(), 4)
    r = p.apply(x) - b
    dv, df = p.dkappa(x, r)
    rng = np.random.default_rng(5)
    h = 1e-6
    for arr, grad, name in ((kv, dv, "vol"), (kf, df, "face")):
        idx = rng.choice(arr.size, 12, replace=False)
        nz = np.flatnonzero(np.abs(grad) > 1e-12)  # include face entries that are active
        idx = np.concatenate([idx, rng.choice(nz, 4, replace=False)])
        for i in idx:
            kp, km = arr.copy(), arr.copy()
            kp[i] += h
            km[i] -= h
            if name == "vol":
                p.kappa_vol = kp; Lp = _loss(p, x, b)
                p.kappa_vol = km; Lm = _loss(p, x, b)
                p.kappa_vol = kv
            else:
                p.kappa_face = kp; Lp = _loss(p, x, b)
                p.kappa_face = km; Lm = _loss(p, x, b)
                p.kappa_face = kf
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])), (name, i, fd, grad[i])


def test_dkappa_sum_identity():
    # A(kappa) is affine in kappa: sum_q kappa_q dL/dkappa_q = r^T A(kappa) x - r^T A(0) x
    p = _trilinear_problem(n=(3, 2, 2), k=2, theta=0.0)
    kv, kf = wl.lognormal_kappa(p.ncell, p.m, seed=2)
    p.kappa_vol, p.kappa_face = kv, kf
    x = wl.uniform_vector(p.ndofs(), 3)
    r = wl.uniform_vector(p.ndofs(), 4)
    dv, df = p.dkappa(x, r)
    full = r @ p.apply(x)
    p.kappa_vol, p.kappa_face = np.zeros_like(kv), np.zeros_like(kf)
    base = r @ p.apply(x)
    assert abs(kv @ dv + kf @ df - (full - base)) < 1e-12 * abs(full)


# ------------------------------------------------------------ data terms (right-hand side)

def _qp_values(v, n, k, func):
    """func at the volume Gauss points [ncell][m^3] and at each cell's face Gauss points
    [ncell][6][m^2] (numpy Gauss nodes, test-side trilinear map)."""
    m = k + 1
    t, _ = npleg.leggauss(m)
    s = (t + 1) / 2
    ncell = n[0] * n[1] * n[2]
    fv = np.zeros((ncell, m ** 3))
    gf = np.zeros((ncell, 6, m * m))
    for c in range(ncell):
        V8 = _cell_corners(v, n, c)
        for q2 in range(m):
            for q1 in range(m):
                for q0 in range(m):
                    fv[c, q0 + m * (q1 + m * q2)] = func(_trilinear_point(V8, (s[q0], s[q1], s[q2])))
        for lf in range(6):
            a, side = lf // 2, lf % 2
            t1, t2 = (1, 2) if a == 0 else ((0, 2) if a == 1 else (0, 1))
            for qt in range(m):
                for qs in range(m):
                    xi = [0.0, 0.0, 0.0]
                    xi[a], xi[t1], xi[t2] = float(side), s[qs], s[qt]
                    gf[c, lf, qs + m * qt] = func(_trilinear_point(V8, xi))
    return fv.ravel(), gf.ravel()


@pytest.mark.parametrize("k", [2, 3])
def test_rhs_paper_manufactured_solution_all_cells_affine(k):
    # Sec. 5.2's g = |x|^2 with kappa = 1, c = 1, f = -6 + |x|^2 and the Dirichlet data
    # terms on every boundary face: A g_I = F exactly on every cell of an affine mesh
    n = (3, 4, 3)
    v = wl.unit_cube_vertices(*n)
    p = oracle.Problem(*n, k, c=1.0)
    u = _interpolate(v, n, k, lambda x: float(x @ x))[:, 0, :].ravel()
    fv, gf = _qp_values(v, n, k, lambda x: float(x @ x) - 6.0)
    _, gg = _qp_values(v, n, k, lambda x: float(x @ x))
    res = p.apply(u) - p.rhs(fv, gg)
    assert np.abs(res).max() < 1e-12 * np.abs(p.apply(u)).max()


@pytest.mark.parametrize("k,theta", [(1, -1.0), (2, 1.0), (2, 0.0)])
def test_rhs_linear_solution_all_cells_perturbed(k, theta):
    # u linear, kappa = 1, c = 0, f = 0, g = u: the theta and penalty data terms cancel
    # their counterparts in A u_I point by point, the rest is integrated exactly
    n = (3, 3, 4)
    v = wl.perturbed_vertices(*n, seed=1)
    p = oracle.Problem(*n, k, vertices=v, c=0.0, theta=theta)
    lin = lambda x: 0.3 + 1.1 * x[0] - 0.7 * x[1] + 0.4 * x[2]
    u = _interpolate(v, n, k, lin)[:, 0, :].ravel()
    _, gg = _qp_values(v, n, k, lin)
    Au = p.apply(u)
    res = Au - p.rhs(None, gg)
    assert np.abs(res).max() < 1e-12 * np.abs(Au).max()


@pytest.mark.parametrize("n,k,mask,c", [((3, 2, 4), 2, 0b111111, 1.0), ((1, 3, 2), 3, 0b010110, 0.5),
                                        ((2, 2, 2), 1, 0, 1.0), ((4, 1, 1), 4, 0b101010, 2.0)])
def test_block_jacobi_cell_blocks_are_kronecker_sums(n, k, mask, c):
    # Each cell's diagonal block of the assembled affine matrix must equal the Kronecker
    # sum of the 1D diagonal blocks of the independent Kronecker construction (the
    # separability that fast diagonalisation relies on), and block_jacobi must invert it.
    orc = oracle.Problem(*n, k, dirichlet_mask=mask, c=c)
    A = orc.assemble()
    b = kr.Basis1D(kr.gll_points(k))
    p = k + 1
    M = [kr.mass_1d(b, b, n[a], 1.0 / n[a]).toarray() for a in range(3)]
    S = [kr.sipg_1d(b, n[a], 1.0 / n[a], kr.gamma_axis(k, n[a], 2.0, 0), -1.0, bool(mask >> (2 * a) & 1),
                    bool(mask >> (2 * a + 1) & 1)).toarray() for a in range(3)]
    r = wl.uniform_vector(orc.ndofs(), 5)
    z = orc.block_jacobi(r)

    def blk(X, e):
        return X[e * p:(e + 1) * p, e * p:(e + 1) * p]

    for cell in range(orc.ncell):
        cx, cy, cz = cell % n[0], (cell // n[0]) % n[1], cell // (n[0] * n[1])
        Mx, My, Mz = blk(M[0], cx), blk(M[1], cy), blk(M[2], cz)
        Kc = (np.kron(Mz, np.kron(My, blk(S[0], cx))) + np.kron(Mz, np.kron(blk(S[1], cy), Mx))
              + np.kron(blk(S[2], cz), np.kron(My, Mx)) + c * np.kron(Mz, np.kron(My, Mx)))
        sl = slice(cell * p ** 3, (cell + 1) * p ** 3)
        assert np.abs(A[sl, sl].toarray() - Kc).max() <= 1e-12 * np.abs(Kc).max()
        assert np.abs(Kc @ z[sl] - r[sl]).max() <= 1e-10 * np.abs(r).max()


def test_block_jacobi_inverts_single_cell_columns():
    # for x supported on one cell c, (A x)_c = A_cc x_c, so block_jacobi(A x) returns x on c
    orc = oracle.Problem(3, 3, 2, 2, dirichlet_mask=0b011011)
    A = orc.assemble()
    loc = 27
    for cell in (0, 7, 17):
        x = np.zeros(orc.ndofs())
        x[cell * loc:(cell + 1) * loc] = wl.uniform_vector(loc, cell)
        z = orc.block_jacobi(A @ x)
        assert np.abs(z[cell * loc:(cell + 1) * loc] - x[cell * loc:(cell + 1) * loc]).max() <= 1e-11
    # B = blockdiag(A)^-1 is symmetric for theta = -1
    u, v = wl.uniform_vector(orc.ndofs(), 1), wl.uniform_vector(orc.ndofs(), 2)
    assert abs(u @ orc.block_jacobi(v) - v @ orc.block_jacobi(u)) <= 1e-12 * abs(u @ orc.block_jacobi(v))


@pytest.mark.parametrize("k,c,beta", [(1, 1.0, 2.0), (2, 0.5, -1.5), (3, 0.0, 4.0)])
def test_semilinear_constant_state_closed_form(k, c, beta):
    # u = a everywhere, no Dirichlet faces: the stiffness and every face term vanish, so
    # the residual r(u) = c a (1, v) + beta a^3 (1, v) sums to (c a + beta a^3) |Omega|,
    # exactly (the integrand is constant), on a perturbed mesh as well
    n = (3, 2, 4)
    orc = oracle.Problem(*n, k, c=c, dirichlet_mask=0, vertices=wl.perturbed_vertices(*n, seed=1))
    a = 0.7
    y = orc.semilinear(np.full(orc.ndofs(), a), beta)
    assert abs(y.sum() - (c * a + beta * a ** 3)) <= 1e-12


def test_semilinear_jacobian_is_the_derivative_of_the_residual():
    # J(u0) w against the central difference of r(u) = A u + beta (u^3, v): for the cubic
    # reaction the difference is exact up to beta eps^2 (w^3, v)
    n, k, beta, eps = (3, 3, 2), 2, 3.0, 1e-4
    orc = oracle.Problem(*n, k, vertices=wl.perturbed_vertices(*n, seed=1))
    u0, w = wl.uniform_vector(orc.ndofs(), 1), wl.uniform_vector(orc.ndofs(), 2)
    J = orc.semilinear(w, beta, u0=u0)
    fd = (orc.semilinear(u0 + eps * w, beta) - orc.semilinear(u0 - eps * w, beta)) / (2 * eps)
    assert np.abs(J - fd).max() <= 1e-7 * np.abs(J).max()
    # beta = 0 reduces both to the linear apply
    assert np.abs(orc.semilinear(w, 0.0) - orc.apply(w)).max() == 0.0
    assert np.abs(orc.semilinear(w, 0.0, u0=u0) - orc.apply(w)).max() == 0.0


@pytest.mark.parametrize("n,degrees,theta,c,mask,pen_mode", [
    ((2, 3, 2), (1, 3, 2), -1.0, 1.0, 0b111111, 0),
    ((3, 2, 2), (4, 1, 2), 1.0, 0.5, 0b100101, 0),
    ((2, 2, 3), (2, 2, 5), -1.0, 0.0, 0b011011, 1),
    ((1, 2, 2), (3, 2, 1), 0.0, 2.0, 0, 0),
])
def test_anisotropic_affine_matches_kronecker(n, degrees, theta, c, mask, pen_mode):
    # per-direction degrees (Sec. 2.1's vector k) against the independent Kronecker
    # construction with one 1D basis per direction
    orc = oracle.Problem(*n, max(degrees), theta=theta, c=c, dirichlet_mask=mask, pen_mode=pen_mode,
                         degrees=degrees)
    A = orc.assemble().toarray()
    K = kr.scalar_matrix(*n, max(degrees), c=c, theta=theta, mask=mask, pen_mode=pen_mode,
                         degrees=degrees).toarray()
    assert A.shape == K.shape == (np.prod(n) * np.prod([d + 1 for d in degrees]),) * 2
    assert np.abs(A - K).max() <= 1e-12 * np.abs(K).max()
    x = wl.uniform_vector(A.shape[0], 0)
    assert np.abs(orc.apply(x) - K @ x).max() <= 1e-12 * np.abs(K @ x).max()


def test_anisotropic_with_equal_degrees_is_the_isotropic_operator_on_a_perturbed_mesh():
    n, k = (3, 2, 3), 2
    verts = wl.perturbed_vertices(*n, seed=1)
    x = wl.uniform_vector(np.prod(n) * (k + 1) ** 3, 0)
    iso = oracle.Problem(*n, k, vertices=verts).apply(x)
    ani = oracle.Problem(*n, k, vertices=verts, degrees=(k, k, k)).apply(x)
    assert np.abs(iso - ani).max() == 0.0


@pytest.mark.parametrize("n,degrees,quad,theta,mask", [
    ((2, 3, 2), (1, 3, 2), (3, 4, 3), -1.0, 0b111111),
    ((3, 2, 2), (2, 2, 2), (4, 3, 5), 1.0, 0b100101),
    ((2, 2, 2), (3, 1, 2), (4, 4, 6), 0.0, 0b011011),
])
def test_anisotropic_quadrature_affine_matches_kronecker(n, degrees, quad, theta, mask):
    # m_a Gauss points per direction, chosen apart from k_a + 1 (Sec. 2.1's tensor-product
    # rule; Sec. 4 raises m on purpose): every integrand of an affine cell is a polynomial
    # that m_a >= k_a + 1 points integrate exactly, so the operator must still equal the
    # exactly integrated Kronecker construction
    orc = oracle.Problem(*n, max(degrees), theta=theta, dirichlet_mask=mask, degrees=degrees, quad=quad)
    A = orc.assemble().toarray()
    K = kr.scalar_matrix(*n, max(degrees), theta=theta, mask=mask, degrees=degrees).toarray()
    assert np.abs(A - K).max() <= 1e-12 * np.abs(K).max()


def _aniso_kappa_linear(n, quad):
    """kappa = 1 + x + 2y + 3z at the volume and face Gauss points of the affine lattice,
    in the per-direction layouts (points from numpy's Gauss-Legendre rule)."""
    nx, ny, nz = n
    s = [(np.polynomial.legendre.leggauss(m)[0] + 1) / 2 for m in quad]
    kv, kf = [], []
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                c0 = np.array([cx / nx, cy / ny, cz / nz])
                h = np.array([1 / nx, 1 / ny, 1 / nz])
                for q2 in range(quad[2]):
                    for q1 in range(quad[1]):
                        for q0 in range(quad[0]):
                            x = c0 + h * np.array([s[0][q0], s[1][q1], s[2][q2]])
                            kv.append(1 + x[0] + 2 * x[1] + 3 * x[2])
                for lf in range(6):
                    a, side = lf // 2, lf % 2
                    t1, t2 = (1, 2) if a == 0 else ((0, 2) if a == 1 else (0, 1))
                    for qt in range(quad[t2]):
                        for qs in range(quad[t1]):
                            xi = np.zeros(3)
                            xi[a], xi[t1], xi[t2] = side, s[t1][qs], s[t2][qt]
                            x = c0 + h * xi
                            kf.append(1 + x[0] + 2 * x[1] + 3 * x[2])
    return np.array(kv), np.array(kf)


def test_anisotropic_quadrature_with_linear_kappa_is_independent_of_the_rule():
    # with kappa linear in x, every integrand of an affine cell is still a polynomial of
    # degree <= 2 m_a - 1 per direction, so two rules with m_a >= k_a + 1 give the same
    # operator; kappa values sit in the per-direction layouts, so a mis-indexed point or
    # face would change the result
    n, degrees = (2, 3, 2), (2, 1, 3)
    x = wl.uniform_vector(np.prod(n) * np.prod([d + 1 for d in degrees]), 3)
    ys = []
    for quad in ((3, 2, 4), (4, 4, 5), (5, 3, 6)):
        kv, kf = _aniso_kappa_linear(n, quad)
        orc = oracle.Problem(*n, 3, degrees=degrees, quad=quad, kappa_vol=kv, kappa_face=kf, theta=1.0)
        ys.append(orc.apply(x))
    for y in ys[1:]:
        assert np.abs(y - ys[0]).max() <= 1e-12 * np.abs(ys[0]).max()
    # and kappa really enters: a constant kappa = 1 gives a different operator
    plain = oracle.Problem(*n, 3, degrees=degrees, quad=(3, 2, 4), theta=1.0).apply(x)
    assert np.abs(plain - ys[0]).max() > 1e-3 * np.abs(ys[0]).max()


def test_anisotropic_quadrature_penalty_closed_form_on_a_perturbed_mesh():
    # u = 1: interior jumps and gradients vanish, so 1^T A 1 = c |Omega| + sum over Dirichlet
    # boundary faces of gamma_F |F|, gamma_a = alpha k_a (k_a + 1) n_a with k_a the degree
    # along the normal; exact for any m_a >= 2 because detJ has degree <= 2 per direction and
    # the boundary faces stay planar
    n, degrees, quad = (3, 2, 3), (1, 3, 2), (2, 5, 3)
    orc = oracle.Problem(*n, 3, degrees=degrees, quad=quad, vertices=wl.perturbed_vertices(*n, seed=1), c=1.5)
    one = np.ones(orc.ndofs())
    want = 1.5 + sum(2 * 2.0 * degrees[a] * (degrees[a] + 1) * n[a] for a in range(3))
    assert abs(one @ orc.apply(one) - want) <= 1e-11 * want


def test_stokes_transpose_equals_assembled_transpose():
    # theta = +1 makes the viscous block non-symmetric; the pressure coupling [[., B^T], [B, 0]]
    # is its own transpose, so A^T swaps the viscous face coefficients only
    p = oracle.Problem(2, 3, 2, 3, problem="stokes", theta=1.0, dirichlet_mask=0b111101)
    A = p.assemble()
    x = wl.uniform_vector(p.ndofs(), 1)
    yt = p.apply(x, transpose=True)
    np.testing.assert_allclose(yt, A.T @ x, rtol=0, atol=1e-13 * abs(yt).max())
    assert abs(A - A.T).max() > 1e-3 * abs(A).max()
