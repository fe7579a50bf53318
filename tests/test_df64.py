"""Double-float variant of the FP64 operator (DG_VARIANT_DF64: the three apply kernels in
pairs-of-FP32 arithmetic with FP64 vectors) through the C ABI, against the oracle at the
FP64 bound and against the FP64 variant."""
import numpy as np
import pytest

import oracle
from paper_1812_08075_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1812_08075_gb300 import build as libbuild, dg  # noqa: E402

libbuild.build()

# The FP64 bound. Double-float carries about 48 significant bits (unit roundoff
# u = 2^-48, 3.6e-15). Each output of the apply passes through about 15 contractions of
# at most 7 terms (interpolation, gradient, metric, transposed derivative, face terms,
# transposed interpolation), each term adding a few u of its own magnitude, so the error
# relative to max |y| is at most about 15 * 7 * 3 u = 1.1e-12 in the worst case and a
# few 1e-14 in practice (measured 0.6e-14 to 4e-14).
TOL64 = 1e-12
# double-float against the FP64 variant: the same sums, a quarter of the worst case
TOL_DF_VS_FP64 = 3e-13


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def df_operator(n, k, geom, nrhs=1, **kw):
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    op = dg.Operator(dg.Mesh(*n, verts), k, max_rhs=nrhs, **kw)
    op.set_variant(dg.DG_VARIANT_DF64)
    assert op.stats().variant == dg.DG_VARIANT_DF64
    return op, verts


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_df64_matches_oracle(k, geom):
    n = (4, 3, 5)
    op, verts = df_operator(n, k, geom)
    x = wl.uniform_vector(op.ndofs, 0)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    err = relerr(y, oracle.Problem(*n, k, vertices=verts).apply(x))
    print(f"df64 Q{k} {geom}: rel err vs oracle {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("mask,theta,c", [(0, -1.0, 1.0), (0b100110, 1.0, 0.0), (0b010101, 0.0, 2.5)])
def test_df64_masks_theta_reaction_and_rhs(mask, theta, c):
    n, k, nrhs = (5, 4, 3), 2, 3
    op, _ = df_operator(n, k, "trilinear", nrhs=nrhs, dirichlet_mask=mask, theta=theta, c=c)
    orc = oracle.Problem(*n, k, vertices=wl.perturbed_vertices(*n, seed=1), dirichlet_mask=mask, theta=theta, c=c)
    xs = np.stack([wl.uniform_vector(op.ndofs, r) for r in range(nrhs)])
    y = op.apply(torch.from_numpy(xs).cuda()).cpu().numpy()
    for r in range(nrhs):
        assert relerr(y[r], orc.apply(xs[r])) <= TOL64


def test_df64_config2_full_size_sampled():
    # 64^3 trilinear Q3, the benchmark workload, on 96 sampled cells
    n, k = (64, 64, 64), 3
    op, verts = df_operator(n, k, "trilinear")
    x = wl.uniform_vector(op.ndofs, 0)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy().reshape(op.mesh.ncell, -1)
    cells = wl.sample_cells(op.mesh.ncell, 96, seed=10)
    ref = oracle.Problem(*n, k, vertices=verts).apply_cells(x, cells, nthreads=0)
    err = float(np.abs(y[cells] - ref).max() / np.abs(ref).max())
    print(f"df64 64^3 Q3 trilinear, sampled cells: rel err {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("k", [2, 3, 5])
def test_df64_agrees_with_fp64_variant(k):
    n = (24, 20, 18)
    op, _ = df_operator(n, k, "trilinear")
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 3)).cuda()
    y_df = op.apply(x)
    op.set_variant(dg.DG_VARIANT_THREE_KERNEL)
    y64 = op.apply(x)
    err = float((y_df - y64).abs().max() / y64.abs().max())
    print(f"df64 vs FP64 Q{k}: {err:.2e}")
    assert err <= TOL_DF_VS_FP64


def test_df64_blockings_and_autotune_keep_the_variant():
    n, k = (12, 10, 9), 3
    op, verts = df_operator(n, k, "trilinear")
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 1)).cuda()
    ref = oracle.Problem(*n, k, vertices=verts).apply(x.cpu().numpy())
    for cpb, fpb in [(1, 2), (2, 64), (8, 16)]:
        op.set_variant(dg.DG_VARIANT_DF64, cpb, fpb)
        assert relerr(op.apply(x).cpu().numpy(), ref) <= TOL64
    res = op.autotune(nrhs=1)
    assert res["variant"] == dg.DG_VARIANT_DF64 and op.stats().variant == dg.DG_VARIANT_DF64
    assert relerr(op.apply(x).cpu().numpy(), ref) <= TOL64


def test_df64_cg_solve():
    # CG with the double-float operator reaches the FP64 target like the FP64 operator
    n, k, nrhs = (6, 5, 7), 2, 2
    b = torch.from_numpy(wl.refinement_rhs(*n, (k + 1) ** 3, seeds=range(nrhs))).cuda()
    its = {}
    for v in (dg.DG_VARIANT_THREE_KERNEL, dg.DG_VARIANT_DF64):
        op = dg.Operator(dg.Mesh(*n), k, max_rhs=nrhs)
        op.set_variant(v)
        x = torch.zeros_like(b)
        ok, info = dg.dg_cg_solve(op.handle, b.data_ptr(), x.data_ptr(), nrhs,
                                  dg.dg_cg_options(1e-10, 5000, 20, 1, dg.DG_PRECOND_NONE), None)
        assert ok
        its[v] = max(i["iters"] for i in info)
        A = oracle.Problem(*n, k).assemble()
        for r in range(nrhs):
            bn, xn = b[r].cpu().numpy(), x[r].cpu().numpy()
            assert np.linalg.norm(bn - A @ xn) <= 1.01e-10 * np.linalg.norm(bn)
    assert abs(its[dg.DG_VARIANT_DF64] - its[dg.DG_VARIANT_THREE_KERNEL]) <= 2


@pytest.mark.parametrize("k,n,mask,theta,mu,nrhs", [(2, (3, 2, 4), 0b111101, -1.0, 1.0, 1),
                                                   (3, (4, 3, 2), 0b010110, 1.0, 0.7, 2),
                                                   (4, (2, 3, 2), 0, -1.0, 2.5, 1), (5, (2, 2, 3), 0b111111, 0.0, 1.0, 1)])
def test_df64_stokes_matches_oracle(k, n, mask, theta, mu, nrhs):
    op = dg.Operator(dg.Mesh(*n), k, problem=dg.DG_STOKES, mu=mu, theta=theta, dirichlet_mask=mask, max_rhs=nrhs)
    op.set_variant(dg.DG_VARIANT_DF64)
    assert op.stats().variant == dg.DG_VARIANT_DF64
    orc = oracle.Problem(*n, k, problem="stokes", mu=mu, theta=theta, dirichlet_mask=mask)
    xs = np.stack([wl.uniform_vector(op.ndofs, 20 + r) for r in range(nrhs)])
    y = op.apply(torch.from_numpy(xs)[0 if nrhs == 1 else slice(None)].cuda()).cpu().numpy().reshape(nrhs, -1)
    err = max(relerr(y[r], orc.apply(xs[r])) for r in range(nrhs))
    print(f"df64 Stokes Q{k}/Q{k - 1}: rel err vs oracle {err:.2e}")
    assert err <= TOL64


def test_df64_stokes_agrees_with_fp64_variant():
    op = dg.Operator(dg.Mesh(16, 16, 16), 3, problem=dg.DG_STOKES)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 4)).cuda()
    y64 = op.apply(x)
    op.set_variant(dg.DG_VARIANT_DF64)
    err = float((op.apply(x) - y64).abs().max() / y64.abs().max())
    print(f"df64 vs FP64 Stokes Q3/Q2 at 16^3: {err:.2e}")
    assert err <= TOL_DF_VS_FP64


def kappa_setup(n, k, geom, theta=-1.0, mask=0b111111, geometry=None):
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    kw = {} if geometry is None else {"geometry": geometry}
    op = dg.Operator(dg.Mesh(*n, verts), k, theta=theta, dirichlet_mask=mask, **kw)
    orc = oracle.Problem(*n, k, vertices=verts, theta=theta, dirichlet_mask=mask)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    orc.kappa_vol, orc.kappa_face = kv, kf
    op._kappa = (torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    op.set_kappa(*op._kappa)
    op.set_variant(dg.DG_VARIANT_DF64)
    assert op.stats().variant == dg.DG_VARIANT_DF64
    return op, orc, kv, kf


@pytest.mark.parametrize("k", [1, 3, 5])
@pytest.mark.parametrize("geometry", [dg.DG_GEOM_STORED, dg.DG_GEOM_RECOMPUTE])
def test_df64_kappa_and_recomputed_geometry_match_oracle(k, geometry):
    n = (4, 3, 5)
    op, orc, _, _ = kappa_setup(n, k, "trilinear", geometry=geometry)
    x = wl.uniform_vector(op.ndofs, 5)
    err = relerr(op.apply(torch.from_numpy(x).cuda()).cpu().numpy(), orc.apply(x))
    print(f"df64 Q{k} trilinear, kappa, geometry {geometry}: rel err {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
@pytest.mark.parametrize("theta", [-1.0, 1.0])
def test_df64_adjoint_and_dkappa_match_oracle(k, geom, theta):
    # y = A^T r and r^T dA/dkappa_q x at every volume and face point, double-float kernels
    n = (4, 3, 5)
    op, orc, kv, kf = kappa_setup(n, k, geom, theta=theta, mask=0b101111)
    x, r = wl.uniform_vector(op.ndofs, 3), wl.uniform_vector(op.ndofs, 4)
    xd, rd = torch.from_numpy(x).cuda(), torch.from_numpy(r).cuda()
    y = torch.empty_like(xd)
    dkv = torch.empty(kv.size, dtype=torch.float64, device="cuda")
    dkf = torch.empty(kf.size, dtype=torch.float64, device="cuda")
    dg.dg_apply_adjoint(op.handle, rd.data_ptr(), xd.data_ptr(), y.data_ptr(), dkv.data_ptr(), dkf.data_ptr(), None, nrhs=1)
    torch.cuda.synchronize()
    rv, rf = orc.dkappa(x, r)
    errs = (relerr(y.cpu().numpy(), orc.apply(r, transpose=True)), relerr(dkv.cpu().numpy(), rv),
            relerr(dkf.cpu().numpy(), rf))
    print(f"df64 adjoint Q{k} {geom} theta {theta}: A^T r {errs[0]:.2e}, dkappa vol {errs[1]:.2e}, face {errs[2]:.2e}")
    assert max(errs) <= TOL64


@pytest.mark.parametrize("k", [2, 3])
def test_df64_semilinear_matches_oracle(k):
    n = (4, 3, 5)
    op, orc, _, _ = kappa_setup(n, k, "trilinear")
    w, u0 = wl.uniform_vector(op.ndofs, 0), wl.uniform_vector(op.ndofs, 1)
    wd, ud = torch.from_numpy(w).cuda(), torch.from_numpy(u0).cuda()
    er = relerr(op.semilinear(wd, 2.5).cpu().numpy(), orc.semilinear(w, 2.5))
    ej = relerr(op.semilinear(wd, 2.5, u0=ud).cpu().numpy(), orc.semilinear(w, 2.5, u0=u0))
    print(f"df64 semilinear Q{k}: residual {er:.2e}, Jacobian {ej:.2e}")
    assert er <= TOL64 and ej <= TOL64


def test_df64_adjoint_agrees_with_fp64_at_config5_scale():
    # 32^3 trilinear Q3 with log-normal kappa: A^T r and dkappa of both variants
    n, k = (32, 32, 32), 3
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), k)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    tk = (torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    op.set_kappa(*tk)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 3)).cuda()
    r = torch.from_numpy(wl.uniform_vector(op.ndofs, 4)).cuda()
    out = {}
    for v in (dg.DG_VARIANT_THREE_KERNEL, dg.DG_VARIANT_DF64):
        op.set_variant(v)
        y = torch.empty_like(x)
        dkv, dkf = torch.empty_like(tk[0]), torch.empty_like(tk[1])
        dg.dg_apply_adjoint(op.handle, r.data_ptr(), x.data_ptr(), y.data_ptr(), dkv.data_ptr(), dkf.data_ptr(), None, nrhs=1)
        out[v] = (y, dkv, dkf)
    a, b = out[dg.DG_VARIANT_THREE_KERNEL], out[dg.DG_VARIANT_DF64]
    errs = [float((q - p).abs().max() / p.abs().max()) for p, q in zip(a, b)]
    print(f"df64 vs FP64 adjoint at 32^3 Q3: y {errs[0]:.2e}, dkappa vol {errs[1]:.2e}, face {errs[2]:.2e}")
    assert max(errs) <= TOL_DF_VS_FP64


def test_df64_where_it_does_not_apply():
    for op in (dg.Operator(dg.Mesh(3, 3, 3), 2, precision=dg.DG_FP32),
               dg.Operator(dg.Mesh(3, 3, 3), 3, problem=dg.DG_STOKES, precision=dg.DG_FP32)):
        with pytest.raises(dg.DGError) as e:
            op.set_variant(dg.DG_VARIANT_DF64)
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
