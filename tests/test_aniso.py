"""Anisotropic degrees and quadrature (Sec. 2.1's vector k and per-direction Gauss rules)
through the C ABI: the run-time-extent three-kernel apply against the oracle's full-basis
evaluation on affine and trilinear-perturbed meshes with and without per-point kappa,
against the isotropic operator for equal degrees, and inside an unpreconditioned CG solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from paper_1812_08075_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1812_08075_gb300 import build as libbuild, dg  # noqa: E402

libbuild.build()

TOL64, TOL32 = 1e-12, 1e-5


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def run(n, degrees, precision=dg.DG_FP64, nrhs=1, quad=None, geom="affine", kappa=False, **kw):
    okw = {k: v for k, v in kw.items() if k in ("c", "theta")}
    if "dirichlet_mask" in kw:
        okw["dirichlet_mask"] = kw["dirichlet_mask"]
    if "penalty_mode" in kw:
        okw["pen_mode"] = kw["penalty_mode"]
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    op = dg.Operator(dg.Mesh(*n, verts), 0, precision=precision, max_rhs=nrhs, degrees=degrees, quad=quad, **kw)
    orc = oracle.Problem(*n, max(degrees), degrees=degrees, quad=quad, vertices=verts, **okw)
    if kappa:
        kv, kf = wl.lognormal_kappa_aniso(op.mesh.ncell, quad or tuple(d + 1 for d in degrees), seed=2)
        orc.kappa_vol, orc.kappa_face = kv, kf
        op.set_kappa(torch.from_numpy(kv).to("cuda", op.dtype), torch.from_numpy(kf).to("cuda", op.dtype))
    assert op.ndofs == orc.ndofs() == np.prod(n) * np.prod([d + 1 for d in degrees])
    xs = np.stack([wl.uniform_vector(op.ndofs, 10 + r) for r in range(nrhs)])
    y = op.apply(torch.from_numpy(xs).to("cuda", op.dtype)).double().cpu().numpy().reshape(nrhs, -1)
    return max(relerr(y[r], orc.apply(xs[r])) for r in range(nrhs))


@pytest.mark.parametrize("geom", ["affine", "trilinear"])
@pytest.mark.parametrize("kappa", [False, True])
@pytest.mark.parametrize("degrees,quad", [((1, 3, 2), (3, 4, 3)), ((3, 4, 3), (4, 6, 5)), ((2, 2, 2), (3, 5, 4)),
                                          ((5, 1, 2), (6, 2, 3)), ((2, 3, 1), None)])
def test_aniso_quadrature_geometry_kappa_fp64(degrees, quad, geom, kappa):
    """Per-direction degrees and Gauss rules (m_a >= k_a + 1, m_a apart from k_a + 1) on a
    ragged mesh, affine or with perturbed interior vertices (geometry recomputed at every
    point), with and without log-normal kappa at every point."""
    err = run((4, 3, 5), degrees, quad=quad, geom=geom, kappa=kappa, theta=1.0, dirichlet_mask=0b101101)
    print(f"anisotropic k={degrees} m={quad} {geom} kappa={kappa}: rel err {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_aniso_quadrature_fp32(geom):
    err = run((5, 4, 3), (1, 3, 2), precision=dg.DG_FP32, nrhs=2, quad=(3, 4, 3), geom=geom, kappa=True)
    print(f"anisotropic FP32 {geom}: rel err {err:.2e}")
    assert err <= TOL32


def test_aniso_trilinear_larger_mesh_sampled():
    n, degrees, quad = (24, 20, 16), (1, 3, 2), (3, 4, 3)
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), 0, degrees=degrees, quad=quad)
    kv, kf = wl.lognormal_kappa_aniso(op.mesh.ncell, quad, seed=2)
    op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    x = wl.uniform_vector(op.ndofs, 4)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy().reshape(op.mesh.ncell, -1)
    cells = wl.sample_cells(op.mesh.ncell, 96, seed=9)
    ref = oracle.Problem(*n, 3, degrees=degrees, quad=quad, vertices=verts, kappa_vol=kv,
                         kappa_face=kf).apply_cells(x, cells)
    assert float(np.abs(y[cells] - ref).max() / np.abs(ref).max()) <= TOL64


@pytest.mark.parametrize("degrees", [(1, 3, 2), (4, 1, 2), (2, 2, 5), (5, 4, 3), (1, 1, 4)])
def test_aniso_fp64_matches_oracle(degrees):
    err = run((4, 3, 5), degrees)
    print(f"anisotropic {degrees}: rel err {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("kw", [dict(theta=1.0, dirichlet_mask=0b100101, c=0.5),
                                dict(theta=0.0, dirichlet_mask=0, c=2.0),
                                dict(penalty_mode=dg.DG_PEN_PAPER, dirichlet_mask=0b011110)])
def test_aniso_theta_masks_penalty_and_rhs(kw):
    assert run((3, 4, 2), (2, 1, 3), nrhs=3, **kw) <= TOL64


def test_aniso_fp32():
    err = run((5, 4, 3), (3, 2, 1), precision=dg.DG_FP32, nrhs=2)
    print(f"anisotropic FP32: rel err {err:.2e}")
    assert err <= TOL32


def test_aniso_equal_degrees_is_the_isotropic_operator():
    n, k = (9, 7, 6), 3
    iso = dg.Operator(dg.Mesh(*n), k)
    ani = dg.Operator(dg.Mesh(*n), 0, degrees=(k, k, k))
    x = torch.from_numpy(wl.uniform_vector(iso.ndofs, 2)).cuda()
    assert relerr(ani.apply(x).cpu().numpy(), iso.apply(x).cpu().numpy()) <= TOL64


def test_aniso_larger_mesh_sampled():
    n, degrees = (40, 24, 18), (1, 3, 2)
    op = dg.Operator(dg.Mesh(*n), 0, degrees=degrees)
    x = wl.uniform_vector(op.ndofs, 4)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy().reshape(op.mesh.ncell, -1)
    cells = wl.sample_cells(op.mesh.ncell, 64, seed=9)
    ref = oracle.Problem(*n, 3, degrees=degrees).apply_cells(x, cells)
    assert float(np.abs(y[cells] - ref).max() / np.abs(ref).max()) <= TOL64


def test_aniso_cg_matches_scipy():
    n, degrees, nrhs = (5, 4, 6), (2, 1, 3), 2
    op = dg.Operator(dg.Mesh(*n), 0, degrees=degrees, max_rhs=nrhs)
    b = torch.from_numpy(np.stack([wl.uniform_vector(op.ndofs, s) for s in range(nrhs)])).cuda()
    x = torch.zeros_like(b)
    ok, info = dg.dg_cg_solve(op.handle, b.data_ptr(), x.data_ptr(), nrhs, dg.dg_cg_options(1e-10, 5000, 20, 1, 0),
                              None)
    assert ok
    A = oracle.Problem(*n, 3, degrees=degrees).assemble()
    bn = b.cpu().numpy()
    for r in range(nrhs):
        got = x[r].cpu().numpy()
        assert np.linalg.norm(bn[r] - A @ got) <= 1.01e-10 * np.linalg.norm(bn[r])
        assert np.abs(got - spla.spsolve(A.tocsc(), bn[r])).max() <= 1e-7 * np.abs(got).max()


def test_aniso_rejections():
    with pytest.raises(dg.DGError) as e:  # the paper's penalty on a trilinear mesh
        dg.Operator(dg.Mesh(3, 3, 3, wl.perturbed_vertices(3, 3, 3)), 0, degrees=(1, 2, 3),
                    penalty_mode=dg.DG_PEN_PAPER, penalty_alpha=3.0)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as e:
        dg.Operator(dg.Mesh(3, 3, 3), 0, degrees=(1, 6, 2))
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    with pytest.raises(dg.DGError) as e:  # fewer Gauss points than k_a + 1
        dg.Operator(dg.Mesh(3, 3, 3), 0, degrees=(1, 3, 2), quad=(2, 3, 3))
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    with pytest.raises(dg.DGError) as e:  # more than 7 points per direction
        dg.Operator(dg.Mesh(3, 3, 3), 0, degrees=(1, 3, 2), quad=(2, 8, 3))
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    op = dg.Operator(dg.Mesh(3, 3, 3), 0, degrees=(1, 2, 3))
    r = torch.ones(op.ndofs, dtype=torch.float64, device="cuda")
    for call in (lambda: op.block_jacobi(r), lambda: op.semilinear(r, 1.0), lambda: op.autotune(),
                 lambda: op.set_variant(dg.DG_VARIANT_THREE_KERNEL, 4, 4)):
        with pytest.raises(dg.DGError) as e:
            call()
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
