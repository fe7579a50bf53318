"""Semilinear reaction through the C ABI: the residual operator A w + beta (w^3, v) and its
Jacobian action A w + 3 beta (u0^2 w, v) (u0 and w evaluated together in one kernel),
against the oracle's full-basis evaluation, and the Jacobian against central differences
of the GPU residual."""
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

TOL64 = 1e-12


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def setup(n, k, geom, kappa, mask=0b111111, theta=-1.0):
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    op = dg.Operator(dg.Mesh(*n, verts), k, dirichlet_mask=mask, theta=theta)
    orc = oracle.Problem(*n, k, vertices=verts, dirichlet_mask=mask, theta=theta)
    if kappa:
        kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
        op._kappa = (torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
        op.set_kappa(*op._kappa)
        orc.kappa_vol, orc.kappa_face = kv, kf
    return op, orc


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_semilinear_residual_and_jacobian_match_oracle(k, geom):
    op, orc = setup((4, 3, 5), k, geom, kappa=(k == 3))
    beta = 2.5
    w, u0 = wl.uniform_vector(op.ndofs, 0), wl.uniform_vector(op.ndofs, 1)
    wd, ud = torch.from_numpy(w).cuda(), torch.from_numpy(u0).cuda()
    r = op.semilinear(wd, beta).cpu().numpy()
    J = op.semilinear(wd, beta, u0=ud).cpu().numpy()
    er, ej = relerr(r, orc.semilinear(w, beta)), relerr(J, orc.semilinear(w, beta, u0=u0))
    print(f"semilinear Q{k} {geom}: residual {er:.2e}, Jacobian {ej:.2e}")
    assert er <= TOL64 and ej <= TOL64


@pytest.mark.parametrize("mask,theta", [(0, -1.0), (0b100110, 1.0)])
def test_semilinear_masks_theta(mask, theta):
    op, orc = setup((3, 4, 3), 2, "trilinear", kappa=False, mask=mask, theta=theta)
    w, u0 = wl.uniform_vector(op.ndofs, 3), wl.uniform_vector(op.ndofs, 4)
    J = op.semilinear(torch.from_numpy(w).cuda(), -1.5, u0=torch.from_numpy(u0).cuda()).cpu().numpy()
    assert relerr(J, orc.semilinear(w, -1.5, u0=u0)) <= TOL64


def test_semilinear_beta_zero_is_the_linear_apply():
    op, _ = setup((5, 4, 3), 3, "trilinear", kappa=True)
    w = torch.from_numpy(wl.uniform_vector(op.ndofs, 5)).cuda()
    y = op.apply(w)
    assert relerr(op.semilinear(w, 0.0).cpu().numpy(), y.cpu().numpy()) <= TOL64
    assert relerr(op.semilinear(w, 0.0, u0=w).cpu().numpy(), y.cpu().numpy()) <= TOL64


def test_semilinear_jacobian_is_the_derivative_of_the_residual_on_the_gpu():
    # central differences of the GPU residual at 16^3 Q3 trilinear: exact up to
    # beta eps^2 (w^3, v) for the cubic reaction
    op, _ = setup((16, 16, 16), 3, "trilinear", kappa=True)
    beta, eps = 3.0, 1e-4
    u0 = torch.from_numpy(wl.uniform_vector(op.ndofs, 6)).cuda()
    w = torch.from_numpy(wl.uniform_vector(op.ndofs, 7)).cuda()
    J = op.semilinear(w, beta, u0=u0)
    fd = (op.semilinear(u0 + eps * w, beta) - op.semilinear(u0 - eps * w, beta)) / (2 * eps)
    err = float((J - fd).abs().max() / J.abs().max())
    print(f"Jacobian vs central differences: {err:.2e}")
    assert err <= 1e-6


def test_semilinear_argument_errors():
    op, _ = setup((2, 2, 2), 2, "affine", kappa=False)
    w = torch.zeros(op.ndofs, dtype=torch.float64, device="cuda")
    y = torch.empty_like(w)
    with pytest.raises(dg.DGError):  # Jacobian without a linearisation point
        dg._check(dg.lib().dg_apply_semilinear(op.handle, dg.DG_SEMILINEAR_JACOBIAN, 1.0, None, w.data_ptr(),
                                               y.data_ptr(), None), "dg_apply_semilinear")
    with pytest.raises(dg.DGError):  # unknown mode
        dg._check(dg.lib().dg_apply_semilinear(op.handle, 7, 1.0, None, w.data_ptr(), y.data_ptr(), None),
                  "dg_apply_semilinear")
    op32 = dg.Operator(dg.Mesh(2, 2, 2), 2, precision=dg.DG_FP32)
    with pytest.raises(dg.DGError) as e:
        op32.semilinear(torch.zeros(op32.ndofs, device="cuda"), 1.0)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
