"""GPU adjoint of the scalar SIPG apply (dg_apply_adjoint and the autograd wrapper):
y = A^T r against the oracle's transposed apply and its assembled matrix, dL/dkappa
against the oracle's pointwise derivative, and both against central finite differences
(step 1e-6) of L = 0.5 ||A(kappa) x - b||^2 on the full 64^3 Q3 configuration."""
import numpy as np
import pytest

import oracle
from paper_1812_08075_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1812_08075_gb300 import build as libbuild, dg  # noqa: E402
from paper_1812_08075_gb300.autograd import dg_apply as dg_apply_ad  # noqa: E402

libbuild.build()
TOL64 = 1e-12


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def setup(n, k, geom, theta=-1.0, kappa=True, mask=0b111111):
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    op = dg.Operator(dg.Mesh(*n, verts), k, theta=theta, dirichlet_mask=mask)
    orc = oracle.Problem(*n, k, vertices=verts, theta=theta, dirichlet_mask=mask)
    kv = kf = None
    if kappa:
        kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
        orc.kappa_vol, orc.kappa_face = kv, kf
        op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    return op, orc, kv, kf


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
@pytest.mark.parametrize("theta", [-1.0, 1.0])
def test_transpose_and_dkappa_vs_oracle(k, geom, theta):
    n = (4, 3, 5)
    op, orc, kv, kf = setup(n, k, geom, theta=theta, mask=0b101111)
    x = wl.uniform_vector(op.ndofs, 3)
    r = wl.uniform_vector(op.ndofs, 4)
    xd, rd = torch.from_numpy(x).cuda(), torch.from_numpy(r).cuda()
    y = torch.empty_like(xd)
    dkv = torch.empty(kv.size, dtype=torch.float64, device="cuda")
    dkf = torch.empty(kf.size, dtype=torch.float64, device="cuda")
    dg.dg_apply_adjoint(op.handle, rd.data_ptr(), xd.data_ptr(), y.data_ptr(), dkv.data_ptr(), dkf.data_ptr(), None, nrhs=1)
    torch.cuda.synchronize()
    assert relerr(y.cpu().numpy(), orc.apply(r, transpose=True)) <= TOL64
    rv, rf = orc.dkappa(x, r)
    assert relerr(dkv.cpu().numpy(), rv) <= TOL64
    assert relerr(dkf.cpu().numpy(), rf) <= TOL64
    # transpose only (no x): same y
    y2 = torch.empty_like(xd)
    dg.dg_apply_adjoint(op.handle, rd.data_ptr(), None, y2.data_ptr(), None, None, None, nrhs=1)
    assert torch.equal(y, y2)


def test_adjoint_without_kappa_equals_forward_for_sipg():
    op, orc, _, _ = setup((3, 4, 3), 3, "trilinear", kappa=False)
    r = torch.from_numpy(wl.uniform_vector(op.ndofs, 4)).cuda()
    y = torch.empty_like(r)
    dg.dg_apply_adjoint(op.handle, r.data_ptr(), None, y.data_ptr(), None, None, None, nrhs=1)
    fwd = op.apply(r)
    assert relerr(y.cpu().numpy(), fwd.cpu().numpy()) <= TOL64


def test_autograd_gradients_on_8cubed_vs_assembled_matrix():
    # config 5's 8^3 sub-case: trilinear Q3, log-normal kappa, L = 0.5||A x - b||^2
    n, k = (8, 8, 8), 3
    op, orc, kv, kf = setup(n, k, "trilinear")
    x0 = wl.uniform_vector(op.ndofs, 3)
    b = wl.uniform_vector(op.ndofs, 4)
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    tkv = torch.from_numpy(kv).cuda().requires_grad_(True)
    tkf = torch.from_numpy(kf).cuda().requires_grad_(True)
    y = dg_apply_ad(op, x, tkv, tkf)
    L = 0.5 * ((y - torch.from_numpy(b).cuda()) ** 2).sum()
    L.backward()
    A = orc.assemble()
    r = A @ x0 - b
    assert relerr(x.grad.cpu().numpy(), A.T @ r) <= TOL64
    rv, rf = orc.dkappa(x0, r)
    assert relerr(tkv.grad.cpu().numpy(), rv) <= TOL64
    assert relerr(tkf.grad.cpu().numpy(), rf) <= TOL64


def test_finite_differences_full_config5():
    # 64^3 trilinear Q3, kappa log-normal (seed 2), x, b ~ U[-1,1] (seeds 3, 4). The change
    # of L under +-h is formed from y+ - y- so that no large numbers cancel.
    n, k = (64, 64, 64), 3
    op, _, _, _ = setup(n, k, "trilinear", kappa=False)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 3)).cuda()
    b = torch.from_numpy(wl.uniform_vector(op.ndofs, 4)).cuda()
    tkv = torch.from_numpy(kv).cuda()
    tkf = torch.from_numpy(kf).cuda()
    op.set_kappa(tkv, tkf)
    r = op.apply(x) - b
    gx = torch.empty_like(x)
    gkv = torch.empty_like(tkv)
    gkf = torch.empty_like(tkf)
    dg.dg_apply_adjoint(op.handle, r.data_ptr(), x.data_ptr(), gx.data_ptr(), gkv.data_ptr(), gkf.data_ptr(), None, nrhs=1)
    h = 1e-6
    rng = np.random.default_rng(9)

    def dL(yp, ym):
        return float(0.5 * ((yp - ym) * (yp + ym - 2 * b)).sum() / (2 * h))

    worst = 0.0
    for idx in rng.choice(op.ndofs, 12, replace=False):
        xp, xm = x.clone(), x.clone()
        xp[idx] += h
        xm[idx] -= h
        fd = dL(op.apply(xp), op.apply(xm))
        g = float(gx[idx])
        worst = max(worst, abs(fd - g) / max(abs(g), 1e-3 * float(gx.abs().max())))
    for arr, grad in ((tkv, gkv), (tkf, gkf)):
        nz = torch.nonzero(grad.abs() > 1e-3 * grad.abs().max()).flatten().cpu().numpy()
        for idx in rng.choice(nz, 12, replace=False):
            kp, km = arr.clone(), arr.clone()
            kp[idx] += h
            km[idx] -= h
            if arr is tkv:
                op.set_kappa(kp, tkf); yp = op.apply(x)
                op.set_kappa(km, tkf); ym = op.apply(x)
            else:
                op.set_kappa(tkv, kp); yp = op.apply(x)
                op.set_kappa(tkv, km); ym = op.apply(x)
            op.set_kappa(tkv, tkf)
            fd = dL(yp, ym)
            g = float(grad[idx])
            worst = max(worst, abs(fd - g) / max(abs(g), 1e-3 * float(grad.abs().max())))
    print(f"worst FD relative error {worst:.2e}")
    assert worst <= 1e-6


# ------------------------------------------- A^T r against finite differences on every config

def fd_gradient_check(op, x, b, idxs, h=1e-6):
    """Largest relative error of dL/dx = A^T (A x - b) from dg_apply_adjoint against central
    differences of L = 0.5 ||A x - b||^2 (formed from y+ - y- so that nothing cancels)."""
    r = op.apply(x) - b
    g = torch.empty_like(x)
    dg.dg_apply_adjoint(op.handle, r.data_ptr(), None, g.data_ptr(), None, None, None, nrhs=1)
    worst = 0.0
    for idx in idxs:
        xp, xm = x.clone(), x.clone()
        xp[idx] += h
        xm[idx] -= h
        yp, ym = op.apply(xp), op.apply(xm)
        fd = float(0.5 * ((yp - ym) * (yp + ym - 2 * b)).sum() / (2 * h))
        gi = float(g[idx])
        worst = max(worst, abs(fd - gi) / max(abs(gi), 1e-3 * float(g.abs().max())))
    return worst


def test_finite_differences_config1():
    op = dg.Operator(dg.Mesh(4, 4, 4), 2)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).cuda()
    b = torch.from_numpy(wl.uniform_vector(op.ndofs, 1)).cuda()
    assert fd_gradient_check(op, x, b, np.random.default_rng(1).choice(op.ndofs, 24, replace=False)) <= 1e-6


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_finite_differences_config2(k):
    n = (64, 64, 64)
    op = dg.Operator(dg.Mesh(*n, wl.perturbed_vertices(*n, seed=1)), k)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).cuda()
    b = torch.from_numpy(wl.uniform_vector(op.ndofs, 1)).cuda()
    assert fd_gradient_check(op, x, b, np.random.default_rng(k).choice(op.ndofs, 6, replace=False)) <= 1e-6


def test_stokes_adjoint_matches_oracle_transpose():
    n, k = (3, 2, 4), 3
    for theta in (-1.0, 1.0):
        op = dg.Operator(dg.Mesh(*n), k, problem=dg.DG_STOKES, dirichlet_mask=0b111101, theta=theta)
        orc = oracle.Problem(*n, k, problem="stokes", dirichlet_mask=0b111101, theta=theta)
        r = wl.uniform_vector(op.ndofs, 2)
        y = torch.empty(op.ndofs, dtype=torch.float64, device="cuda")
        rd = torch.from_numpy(r).cuda()
        dg.dg_apply_adjoint(op.handle, rd.data_ptr(), None, y.data_ptr(), None, None, None, nrhs=1)
        assert relerr(y.cpu().numpy(), orc.apply(r, transpose=True)) <= TOL64


def test_finite_differences_config3_stokes():
    n = (32, 32, 32)
    op = dg.Operator(dg.Mesh(*n), 3, problem=dg.DG_STOKES, dirichlet_mask=0b111101)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).cuda()
    b = torch.from_numpy(wl.uniform_vector(op.ndofs, 1)).cuda()
    rng = np.random.default_rng(3)
    nvel = op.mesh.ncell * 3 * 64
    idxs = np.concatenate([rng.choice(nvel, 8, replace=False), nvel + rng.choice(op.ndofs - nvel, 4, replace=False)])
    assert fd_gradient_check(op, x, b, idxs) <= 1e-6


def test_finite_differences_config4_and_fp32_transpose():
    # 128^3 affine Q2: FD of the FP64 operator's gradient; the FP32 operator's transposed
    # apply (the persistent cellwise kernel with exchanged coefficients) against it at 1e-5
    n = (128, 128, 128)
    op = dg.Operator(dg.Mesh(*n), 2)
    x = torch.from_numpy(wl.refinement_rhs(*n, 27, seeds=[0])[0]).cuda()
    b = torch.from_numpy(wl.uniform_vector(op.ndofs, 1)).cuda()
    assert fd_gradient_check(op, x, b, np.random.default_rng(4).choice(op.ndofs, 6, replace=False)) <= 1e-6
    op32 = dg.Operator(dg.Mesh(*n), 2, precision=dg.DG_FP32)
    r = b
    g64 = torch.empty_like(r)
    dg.dg_apply_adjoint(op.handle, r.data_ptr(), None, g64.data_ptr(), None, None, None, nrhs=1)
    r32 = r.float()
    g32 = torch.empty_like(r32)
    dg.dg_apply_adjoint(op32.handle, r32.data_ptr(), None, g32.data_ptr(), None, None, None, nrhs=1)
    assert float((g32.double() - g64).abs().max() / g64.abs().max()) <= 1e-5


@pytest.mark.parametrize("nrhs", [3, 16])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_multi_rhs_adjoint_vs_oracle(nrhs, geom):
    """nrhs right-hand sides in one call: y_s = A^T r_s per right-hand side against the
    oracle's transposed apply, and dkappa against the oracle's derivative summed over s
    (the gradient of the summed loss)."""
    n, k = (4, 3, 5), 3
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    op = dg.Operator(dg.Mesh(*n, verts), k, theta=1.0, dirichlet_mask=0b101111, max_rhs=nrhs)
    orc = oracle.Problem(*n, k, vertices=verts, theta=1.0, dirichlet_mask=0b101111)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    orc.kappa_vol, orc.kappa_face = kv, kf
    op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    X = np.stack([wl.uniform_vector(op.ndofs, 30 + s) for s in range(nrhs)])
    R = np.stack([wl.uniform_vector(op.ndofs, 60 + s) for s in range(nrhs)])
    xd, rd = torch.from_numpy(X).cuda(), torch.from_numpy(R).cuda()
    y = torch.full_like(xd, float("nan"))
    dkv = torch.full((kv.size,), float("nan"), dtype=torch.float64, device="cuda")
    dkf = torch.full((kf.size,), float("nan"), dtype=torch.float64, device="cuda")
    dg.dg_apply_adjoint(op.handle, rd.data_ptr(), xd.data_ptr(), y.data_ptr(), dkv.data_ptr(), dkf.data_ptr(), None,
                        nrhs=nrhs)
    torch.cuda.synchronize()
    yh = y.cpu().numpy()
    sv, sf = np.zeros(kv.size), np.zeros(kf.size)
    for s in range(nrhs):
        assert relerr(yh[s], orc.apply(R[s], transpose=True)) <= TOL64, s
        rv, rf = orc.dkappa(X[s], R[s])
        sv += rv
        sf += rf
    assert relerr(dkv.cpu().numpy(), sv) <= TOL64
    assert relerr(dkf.cpu().numpy(), sf) <= TOL64


def test_multi_rhs_adjoint_rejects_more_than_max_rhs():
    op = dg.Operator(dg.Mesh(2, 2, 2), 2, max_rhs=2)
    r = torch.zeros(3 * op.ndofs, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(r)
    with pytest.raises(dg.DGError) as e:
        dg.dg_apply_adjoint(op.handle, r.data_ptr(), None, y.data_ptr(), None, None, None, nrhs=3)
    assert e.value.status == dg.DG_ERR_INVALID_ARG


@pytest.mark.parametrize("problem", ["stokes", "fp32"])
def test_multi_rhs_transpose_without_kappa(problem):
    """Stokes and FP32 operators: y_s = A^T r_s for 3 right-hand sides in one call, each
    against the single-vector call (Stokes: and the oracle's transpose)."""
    nrhs = 3
    if problem == "stokes":
        n, k = (3, 2, 3), 3
        op = dg.Operator(dg.Mesh(*n), k, problem=dg.DG_STOKES, dirichlet_mask=0b111101, theta=1.0, max_rhs=nrhs)
        orc = oracle.Problem(*n, k, problem="stokes", dirichlet_mask=0b111101, theta=1.0)
    else:
        n, k = (4, 3, 5), 2
        op = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32, theta=1.0, max_rhs=nrhs)
        orc = None
    R = np.stack([wl.uniform_vector(op.ndofs, 90 + s) for s in range(nrhs)])
    rd = torch.from_numpy(R).to("cuda", op.dtype)
    y = torch.empty_like(rd)
    dg.dg_apply_adjoint(op.handle, rd.data_ptr(), None, y.data_ptr(), None, None, None, nrhs=nrhs)
    for s in range(nrhs):
        ys = torch.empty_like(rd[s])
        dg.dg_apply_adjoint(op.handle, rd[s].data_ptr(), None, ys.data_ptr(), None, None, None, nrhs=1)
        assert torch.equal(ys, y[s]), s
        if orc is not None:
            assert relerr(y[s].cpu().numpy(), orc.apply(R[s], transpose=True)) <= TOL64


def test_autograd_batched_x_sums_dkappa():
    """DGApply with x of shape [nrhs, ndofs]: dL/dx per right-hand side and dL/dkappa summed,
    against the oracle's transposed apply and pointwise derivative."""
    n, k, nrhs = (3, 4, 3), 2, 4
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), k, max_rhs=nrhs)
    orc = oracle.Problem(*n, k, vertices=verts)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    orc.kappa_vol, orc.kappa_face = kv, kf
    X = np.stack([wl.uniform_vector(op.ndofs, 5 + s) for s in range(nrhs)])
    B = np.stack([wl.uniform_vector(op.ndofs, 50 + s) for s in range(nrhs)])
    x = torch.from_numpy(X).cuda().requires_grad_(True)
    tkv = torch.from_numpy(kv).cuda().requires_grad_(True)
    tkf = torch.from_numpy(kf).cuda().requires_grad_(True)
    y = dg_apply_ad(op, x, tkv, tkf)
    loss = 0.5 * ((y - torch.from_numpy(B).cuda()) ** 2).sum()
    loss.backward()
    sv, sf = np.zeros(kv.size), np.zeros(kf.size)
    for s in range(nrhs):
        r = orc.apply(X[s]) - B[s]
        assert relerr(x.grad[s].cpu().numpy(), orc.apply(r, transpose=True)) <= TOL64
        rv, rf = orc.dkappa(X[s], r)
        sv += rv
        sf += rf
    assert relerr(tkv.grad.cpu().numpy(), sv) <= TOL64
    assert relerr(tkf.grad.cpu().numpy(), sf) <= TOL64
