"""GPU data terms of the residual (dg_rhs) against the oracle's load vector, and the
residual r = A u - F of exactly representable solutions computed entirely on the GPU."""
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


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_rhs_matches_oracle(k, geom):
    n = (4, 3, 5)
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    ncell, m = n[0] * n[1] * n[2], k + 1
    f = wl.uniform_vector(ncell * m ** 3, 5)
    g = wl.uniform_vector(ncell * 6 * m * m, 6)
    kv, kf = wl.lognormal_kappa(ncell, m, seed=2)
    for theta, mask, kappa in ((-1.0, 0b111111, False), (1.0, 0b011101, True)):
        op = dg.Operator(dg.Mesh(*n, verts), k, theta=theta, dirichlet_mask=mask)
        orc = oracle.Problem(*n, k, vertices=verts, theta=theta, dirichlet_mask=mask)
        if kappa:
            op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
            orc.kappa_vol, orc.kappa_face = kv, kf
        F = op.rhs(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
        assert relerr(F, orc.rhs(f, g)) <= 1e-12
        F0 = op.rhs(None, torch.from_numpy(g).cuda()).cpu().numpy()
        assert relerr(F0, orc.rhs(None, g)) <= 1e-12


def test_rhs_fp32():
    n, k = (5, 4, 3), 2
    ncell, m = 60, 3
    f = wl.uniform_vector(ncell * m ** 3, 5)
    g = wl.uniform_vector(ncell * 6 * m * m, 6)
    op = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32)
    F = op.rhs(torch.from_numpy(f).float().cuda(), torch.from_numpy(g).float().cuda()).double().cpu().numpy()
    assert relerr(F, oracle.Problem(*n, k).rhs(f, g)) <= 1e-5
