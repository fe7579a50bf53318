"""GPU parity of the DG Stokes block operator (Eq. stokes_weak, Sec. 5.3) against the
CPU oracle, through the C ABI. Vector layout [u: ncell x 3 x (k+1)^3 | p: ncell x k^3];
error metric max|y - y_ref| / max|y_ref|; FP64 to 1e-12, FP32 to 1e-5."""
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
TOL32 = 1e-5
GAMMA_D = 0b111101  # Sec. 5.3: Dirichlet on all faces except x = 1


def run_case(n, k, mask=GAMMA_D, theta=-1.0, mu=1.0, precision=dg.DG_FP64, nrhs=1, seed=0):
    op = dg.Operator(dg.Mesh(*n), k, problem=dg.DG_STOKES, mu=mu, theta=theta, dirichlet_mask=mask,
                     precision=precision, max_rhs=nrhs)
    orc = oracle.Problem(*n, k, problem="stokes", mu=mu, theta=theta, dirichlet_mask=mask)
    assert op.ndofs == orc.ndofs()
    xs = np.stack([wl.uniform_vector(op.ndofs, seed + r) for r in range(nrhs)])
    xd = torch.from_numpy(xs).to("cuda", op.dtype)
    y = op.apply(xd if nrhs > 1 else xd[0]).double().cpu().numpy().reshape(nrhs, -1)
    errs = []
    for r in range(nrhs):
        ref = orc.apply(xs[r])
        errs.append(float(np.abs(y[r] - ref).max() / np.abs(ref).max()))
    return max(errs)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_stokes_degrees_ragged_mesh(k):
    assert run_case((3, 2, 4), k) <= TOL64


@pytest.mark.parametrize("mask,theta,mu", [(0b111111, -1.0, 1.0), (0, -1.0, 2.5), (0b010110, 1.0, 0.7),
                                           (GAMMA_D, 0.0, 1.0)])
def test_stokes_masks_theta_mu(mask, theta, mu):
    assert run_case((4, 3, 2), 3, mask=mask, theta=theta, mu=mu) <= TOL64


def test_stokes_multiple_rhs_and_single_cell():
    assert run_case((2, 3, 2), 3, nrhs=3) <= TOL64
    assert run_case((1, 1, 1), 2) <= TOL64


@pytest.mark.parametrize("k", [2, 3])
def test_stokes_fp32(k):
    err = run_case((4, 3, 3), k, precision=dg.DG_FP32)
    print(f"Stokes FP32 Q{k}: rel err {err:.2e}")
    assert err <= TOL32


def test_stokes_unsupported_cases():
    with pytest.raises(dg.DGError) as e:
        dg.Operator(dg.Mesh(2, 2, 2), 1, problem=dg.DG_STOKES)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as e:
        dg.Operator(dg.Mesh(2, 2, 2, wl.perturbed_vertices(2, 2, 2)), 2, problem=dg.DG_STOKES)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED


# config 3 at full size: 32^3 affine cells, velocity Q3, pressure Q2, sampled cells
def test_config3_full_size_sampled():
    n, k = (32, 32, 32), 3
    op = dg.Operator(dg.Mesh(*n), k, problem=dg.DG_STOKES, dirichlet_mask=GAMMA_D)
    assert op.ndofs == 6291456 + 884736
    x = wl.uniform_vector(op.ndofs, 0)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ncell, P3, PP3 = 32 ** 3, 64, 27
    yu = y[: ncell * 3 * P3].reshape(ncell, 3 * P3)
    yp = y[ncell * 3 * P3:].reshape(ncell, PP3)
    cells = wl.sample_cells(ncell, 96, seed=13)
    ref = oracle.Problem(*n, k, problem="stokes", dirichlet_mask=GAMMA_D).apply_cells(x, cells)
    got = np.concatenate([yu[cells], yp[cells]], axis=1)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert err <= TOL64, err
