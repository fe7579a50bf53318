"""The no-allocation entry point dg_apply_affine_static, called through the C ABI,
against the operator-based dg_apply on the same inputs.

dg_apply_affine_static serves callers that cannot call cudaMalloc (a host framework
that owns all device memory, or loops that must not take cudaMalloc's implicit
synchronisation): its scratch is a fixed 32 MiB device array shared by all calls. The
checks run several calls in a row with different sizes and degrees, so leftovers of one
call in the shared array must not affect the next. This file is collected last.
"""
import numpy as np
import pytest

from paper_1812_08075_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1812_08075_gb300 import build as libbuild, dg  # noqa: E402

libbuild.build()
TOL64 = 1e-12


def _both(n, k, c, theta, alpha, mask, seed):
    op = dg.Operator(dg.Mesh(*n), k, c=c, theta=theta, penalty_alpha=alpha, dirichlet_mask=mask)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, seed)).cuda()
    ref = op.apply(x)
    y = torch.full_like(x, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    dg.dg_apply_affine_static(*n, k, c, theta, alpha, mask, x.data_ptr(), y.data_ptr(), stream)
    torch.cuda.synchronize()
    r, yy = ref.cpu().numpy(), y.cpu().numpy()
    return float(np.abs(yy - r).max() / np.abs(r).max())


def test_static_apply_matches_dg_apply_on_consecutive_calls():
    cases = [((6, 5, 4), 3, 1.0, -1.0, 2.0, 0b111111, 0),
             ((5, 4, 7), 2, 0.5, 1.0, 3.0, 0b101101, 1),
             ((6, 5, 4), 3, 1.0, -1.0, 2.0, 0b111111, 2),
             ((3, 3, 3), 5, 2.0, 0.0, 2.0, 0b010110, 3)]
    for case in cases:
        err = _both(*case)
        assert err <= TOL64, (case, err)


def test_static_apply_rejects_problems_beyond_its_scratch():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as e:
        dg.dg_apply_affine_static(64, 64, 64, 3, 1.0, -1.0, 2.0, 63, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as e:
        dg.dg_apply_affine_static(2, 2, 2, 2, 1.0, -1.0, 2.0, 63, x.data_ptr(), x.data_ptr(), None)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
