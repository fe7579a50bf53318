"""The no-allocation entry point dg_apply_affine_static, called through the C ABI,
against the operator-based dg_apply on the same inputs and against the CPU oracle.

dg_apply_affine_static serves callers that cannot call cudaMalloc (a host framework
that owns all device memory through its own pool, or loops that must not take
cudaMalloc's implicit synchronisation): its scratch is a fixed 32 MiB device array shared
by all calls. The checks run several calls in a row with different sizes and degrees, so
leftovers of one call in the shared array must not affect the next, and they include the
largest problem the array accepts and the first one it rejects. This file is collected
last.
"""
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
SCRATCH = (32 << 20) - 5 * 4096  # bytes of the array left after the five table slots


def _relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _max_cells(k):
    p = k + 1
    return SCRATCH // ((p ** 3 + 24 * p ** 2) * 8)


def _static(n, k, c, theta, alpha, mask, x, stream=None):
    y = torch.full_like(x, float("nan"))
    s = (stream or torch.cuda.current_stream()).cuda_stream
    dg.dg_apply_affine_static(*n, k, c, theta, alpha, mask, x.data_ptr(), y.data_ptr(), s)
    return y


def _case(n, k, c, theta, alpha, mask, seed, stream=None, oracle_cells=None):
    """Relative errors of the static apply against dg_apply and against the oracle (all
    cells, or a sample of them)."""
    op = dg.Operator(dg.Mesh(*n), k, c=c, theta=theta, penalty_alpha=alpha, dirichlet_mask=mask)
    xh = wl.uniform_vector(op.ndofs, seed)
    x = torch.from_numpy(xh).cuda()
    ref = op.apply(x)
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            y = _static(n, k, c, theta, alpha, mask, x, stream)
        torch.cuda.current_stream().wait_stream(stream)
    else:
        y = _static(n, k, c, theta, alpha, mask, x)
    torch.cuda.synchronize()
    yy = y.cpu().numpy()
    err_apply = _relerr(yy, ref.cpu().numpy())
    orc = oracle.Problem(*n, k, c=c, theta=theta, pen_alpha=alpha, dirichlet_mask=mask)
    p3 = (k + 1) ** 3
    if oracle_cells is None:
        err_oracle = _relerr(yy, orc.apply(xh))
    else:
        cells = wl.sample_cells(orc.ncell, oracle_cells, seed=seed + 100)
        got = yy.reshape(-1, p3)[cells].ravel()
        err_oracle = _relerr(got, orc.apply_cells(xh, cells).ravel())
    return err_apply, err_oracle


def test_static_apply_consecutive_calls_all_degrees():
    """Calls of degrees 1..5 and different sizes in a row (the shared array keeps the
    previous call's contents), each against dg_apply and the oracle."""
    cases = [((6, 5, 4), 3, 1.0, -1.0, 2.0, 0b111111, 0),
             ((5, 4, 7), 2, 0.5, 1.0, 3.0, 0b101101, 1),
             ((7, 3, 5), 1, 1.0, -1.0, 2.0, 0b111111, 2),
             ((6, 5, 4), 3, 1.0, -1.0, 2.0, 0b111111, 3),
             ((3, 4, 3), 4, 1.5, 0.0, 2.0, 0b011110, 4),
             ((3, 3, 3), 5, 2.0, 0.0, 2.0, 0b010110, 5)]
    for case in cases:
        ea, eo = _case(*case)
        assert ea <= TOL64 and eo <= TOL64, (case, ea, eo)


def test_static_apply_two_calls_in_a_row_agree():
    n, k = (5, 6, 4), 3
    x = torch.from_numpy(wl.uniform_vector(np.prod(n) * (k + 1) ** 3, 9)).cuda()
    y1 = _static(n, k, 1.0, -1.0, 2.0, 63, x)
    y2 = _static(n, k, 1.0, -1.0, 2.0, 63, x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_static_apply_on_a_non_default_stream():
    ea, eo = _case((4, 5, 6), 2, 1.0, -1.0, 2.0, 0b111111, 6, stream=torch.cuda.Stream())
    assert ea <= TOL64 and eo <= TOL64


def test_static_apply_largest_accepted_and_first_rejected_size():
    """The largest cell count whose scratch fits the array runs (the top of the array is
    used) and matches dg_apply and the oracle on sampled cells; one cell more is
    rejected with DG_ERR_UNSUPPORTED before anything is launched."""
    k = 3
    nmax = _max_cells(k)
    assert nmax == 9356
    ea, eo = _case((nmax, 1, 1), k, 1.0, -1.0, 2.0, 0b111111, 7, oracle_cells=256)
    assert ea <= TOL64 and eo <= TOL64, (ea, eo)
    x = torch.zeros((nmax + 1) * (k + 1) ** 3, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(dg.DGError) as e:
        dg.dg_apply_affine_static(nmax + 1, 1, 1, k, 1.0, -1.0, 2.0, 63, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    # degree 1: the same bound with its own per-cell size
    n1 = _max_cells(1)
    with pytest.raises(dg.DGError) as e:
        dg.dg_apply_affine_static(n1 + 1, 1, 1, 1, 1.0, -1.0, 2.0, 63, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED


def test_static_apply_rejects_bad_arguments():
    x = torch.zeros(2 * 27 * 8, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    bad = [
        (2, 2, 2, 2, x.data_ptr(), x.data_ptr()),             # y is x
        (2, 2, 2, 2, x.data_ptr(), x.data_ptr() + 8 * 64),    # partial overlap (16-byte aligned)
        (2, 2, 2, 2, x.data_ptr() + 8, y.data_ptr()),         # misaligned x
        (0, 2, 2, 2, x.data_ptr(), y.data_ptr()),             # empty mesh
    ]
    for nx, ny, nz, k, xp, yp in bad:
        with pytest.raises(dg.DGError) as e:
            dg.dg_apply_affine_static(nx, ny, nz, k, 1.0, -1.0, 2.0, 63, xp, yp, None)
        assert e.value.status == dg.DG_ERR_INVALID_ARG, (nx, k, xp - x.data_ptr(), yp - x.data_ptr())
    with pytest.raises(dg.DGError) as e:
        dg.dg_apply_affine_static(2, 2, 2, 6, 1.0, -1.0, 2.0, 63, x.data_ptr(), y.data_ptr(), None)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
