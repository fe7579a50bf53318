"""Anisotropic degrees (Sec. 2.1's vector k) through the C ABI: the run-time-extent
three-kernel apply against the oracle's full-basis evaluation, against the isotropic
operator for equal degrees, and inside an unpreconditioned CG solve."""
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


def run(n, degrees, precision=dg.DG_FP64, nrhs=1, **kw):
    okw = {k: v for k, v in kw.items() if k in ("c", "theta")}
    if "dirichlet_mask" in kw:
        okw["dirichlet_mask"] = kw["dirichlet_mask"]
    if "penalty_mode" in kw:
        okw["pen_mode"] = kw["penalty_mode"]
    op = dg.Operator(dg.Mesh(*n), 0, precision=precision, max_rhs=nrhs, degrees=degrees, **kw)
    orc = oracle.Problem(*n, max(degrees), degrees=degrees, **okw)
    assert op.ndofs == orc.ndofs() == np.prod(n) * np.prod([d + 1 for d in degrees])
    xs = np.stack([wl.uniform_vector(op.ndofs, 10 + r) for r in range(nrhs)])
    y = op.apply(torch.from_numpy(xs).to("cuda", op.dtype)).double().cpu().numpy().reshape(nrhs, -1)
    return max(relerr(y[r], orc.apply(xs[r])) for r in range(nrhs))


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
    with pytest.raises(dg.DGError) as e:  # trilinear mesh
        dg.Operator(dg.Mesh(3, 3, 3, wl.perturbed_vertices(3, 3, 3)), 0, degrees=(1, 2, 3))
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as e:
        dg.Operator(dg.Mesh(3, 3, 3), 0, degrees=(1, 6, 2))
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    op = dg.Operator(dg.Mesh(3, 3, 3), 0, degrees=(1, 2, 3))
    r = torch.ones(op.ndofs, dtype=torch.float64, device="cuda")
    for call in (lambda: op.block_jacobi(r), lambda: op.semilinear(r, 1.0), lambda: op.autotune(),
                 lambda: op.set_variant(dg.DG_VARIANT_THREE_KERNEL, 4, 4),
                 lambda: op.set_kappa(torch.ones(27 * 64, dtype=torch.float64, device="cuda"),
                                      torch.ones(27 * 6 * 16, dtype=torch.float64, device="cuda"))):
        with pytest.raises(dg.DGError) as e:
            call()
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
