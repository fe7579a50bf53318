"""GPU cell-block Jacobi preconditioner (fast diagonalisation) through the C ABI, against the
oracle's assembled cell blocks, and inside the batched CG and the refinement solve."""
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

# The apply's bounds: the 1D generalized eigenvectors are exact up to rounding, which the
# cell block's condition number (about 1e3 with the interior penalty) could amplify; the
# measured errors are about 3e-15 (FP64) and 3e-7 (FP32).
TOL64 = 1e-12
TOL32 = 1e-5


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def run(n, k, precision=dg.DG_FP64, nrhs=1, mask=0b111111, c=1.0, alpha=2.0, per_cell=False):
    """Largest relative error of z = blockdiag(A)^-1 r: against the oracle's dense block
    solves, or (per_cell, no assembly) through A_cc z_c = r_c with the oracle's apply of A to
    z restricted to each cell."""
    op = dg.Operator(dg.Mesh(*n), k, precision=precision, max_rhs=nrhs, dirichlet_mask=mask, c=c,
                     penalty_alpha=alpha)
    orc = oracle.Problem(*n, k, dirichlet_mask=mask, c=c, pen_alpha=alpha)
    rs = np.stack([wl.uniform_vector(op.ndofs, 11 + i) for i in range(nrhs)])
    z = op.block_jacobi(torch.from_numpy(rs).to("cuda", op.dtype)).double().cpu().numpy()
    if not per_cell:
        return max(relerr(z[i], orc.block_jacobi(rs[i])) for i in range(nrhs))
    loc, err = (k + 1) ** 3, 0.0
    for i in range(nrhs):
        for cell in range(orc.ncell):
            e = np.zeros(op.ndofs)
            e[cell * loc:(cell + 1) * loc] = z[i, cell * loc:(cell + 1) * loc]
            ac = orc.apply_cells(e, np.array([cell]))[0]
            err = max(err, relerr(ac, rs[i, cell * loc:(cell + 1) * loc]))
    return err


@pytest.mark.parametrize("k,n", [(1, (4, 3, 5)), (2, (4, 3, 5)), (3, (3, 3, 4)), (4, (3, 2, 3)), (5, (2, 3, 2))])
def test_block_jacobi_matches_oracle_fp64(k, n):
    err = run(n, k, per_cell=k >= 4)
    print(f"block Jacobi Q{k}: rel err {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("n,mask,c", [((1, 4, 3), 0b111111, 1.0), ((5, 1, 2), 0b010101, 0.0),
                                      ((3, 3, 3), 0, 1.0), ((2, 5, 1), 0b100110, 3.0)])
def test_block_jacobi_positions_masks_and_thin_meshes(n, mask, c):
    assert run(n, 2, mask=mask, c=c, nrhs=2) <= TOL64


@pytest.mark.parametrize("k", [1, 2, 3])
def test_block_jacobi_fp32(k):
    err = run((5, 4, 3), k, precision=dg.DG_FP32, nrhs=3, per_cell=True)
    print(f"block Jacobi FP32 Q{k}: rel err {err:.2e}")
    assert err <= TOL32


def test_block_jacobi_large_grid_stride():
    # more cell groups than blocks: every block loops over several groups
    n, k = (40, 36, 33), 1
    op = dg.Operator(dg.Mesh(*n), k, max_rhs=2)
    r = torch.from_numpy(np.stack([wl.uniform_vector(op.ndofs, s) for s in (1, 2)])).cuda()
    z = op.block_jacobi(r).cpu().numpy().reshape(2, op.mesh.ncell, 8)
    cells = wl.sample_cells(op.mesh.ncell, 40, seed=3)
    # A_cc z_c = r_c per sampled cell: the oracle's (A e)_c for e = z on cell c and 0 elsewhere
    orc = oracle.Problem(*n, k)
    rn = r.cpu().numpy().reshape(2, op.mesh.ncell, 8)
    for cell in cells:
        zc = np.zeros(op.ndofs)
        zc[cell * 8:(cell + 1) * 8] = z[0, cell]
        Az = orc.apply_cells(zc, np.array([cell]))[0]
        assert np.abs(Az - rn[0, cell]).max() <= 1e-10 * np.abs(rn[0, cell]).max()


def test_block_jacobi_rejected_where_it_does_not_apply():
    cases = [dg.Operator(dg.Mesh(3, 3, 3, wl.perturbed_vertices(3, 3, 3)), 2),
             dg.Operator(dg.Mesh(3, 3, 3), 2, theta=1.0),
             dg.Operator(dg.Mesh(3, 3, 3), 2, quad_points=4)]
    op = dg.Operator(dg.Mesh(3, 3, 3), 2)
    kv, kf = wl.lognormal_kappa(27, 3, seed=2)
    op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    cases.append(op)
    for op in cases:
        r = torch.ones(op.ndofs, dtype=torch.float64, device="cuda")
        with pytest.raises(dg.DGError) as e:
            op.block_jacobi(r)
        assert e.value.status == dg.DG_ERR_UNSUPPORTED


def cg(op, b, rtol, precond, max_iters=5000):
    x = torch.zeros_like(b)
    opt = dg.dg_cg_options(rtol, max_iters, 20, 1, precond)
    ok, info = dg.dg_cg_solve(op.handle, b.data_ptr(), x.data_ptr(), b.shape[0], opt, None)
    return ok, info, x


def test_cg_block_jacobi_converges_in_fewer_iterations():
    n, k, nrhs = (6, 5, 7), 2, 2
    op = dg.Operator(dg.Mesh(*n), k, max_rhs=nrhs)
    b = torch.from_numpy(wl.refinement_rhs(*n, (k + 1) ** 3, seeds=range(nrhs))).cuda()
    ok0, info0, _ = cg(op, b, 1e-10, dg.DG_PRECOND_NONE)
    ok1, info1, x1 = cg(op, b, 1e-10, dg.DG_PRECOND_BLOCK_JACOBI)
    assert ok0 and ok1
    A = oracle.Problem(*n, k).assemble()
    bn = b.cpu().numpy()
    for r in range(nrhs):
        got = x1[r].cpu().numpy()
        assert np.linalg.norm(bn[r] - A @ got) <= 1.01e-10 * np.linalg.norm(bn[r])
        assert np.abs(got - spla.spsolve(A.tocsc(), bn[r])).max() <= 1e-7 * np.abs(got).max()
    it0 = max(i["iters"] for i in info0)
    it1 = max(i["iters"] for i in info1)
    print(f"CG iterations: none {it0}, block Jacobi {it1}")
    assert it1 < it0


def test_refinement_with_block_jacobi_inner_cg():
    n, k, nrhs = (8, 6, 5), 2, 3
    op64 = dg.Operator(dg.Mesh(*n), k, max_rhs=nrhs)
    op32 = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32, max_rhs=nrhs)
    b = torch.from_numpy(wl.refinement_rhs(*n, (k + 1) ** 3, seeds=range(nrhs))).cuda()
    x = torch.zeros_like(b)
    inner = dg.dg_cg_options(1e-3, 2000, 20, 1, dg.DG_PRECOND_BLOCK_JACOBI)
    ok, info = dg.dg_refine_solve(op64.handle, op32.handle, b.data_ptr(), x.data_ptr(), nrhs, 1e-10, 20, inner, None)
    assert ok and all(i["converged"] for i in info)
    A = oracle.Problem(*n, k).assemble()
    bn, xn = b.cpu().numpy(), x.cpu().numpy()
    for r in range(nrhs):
        assert np.linalg.norm(bn[r] - A @ xn[r]) <= 1.01e-10 * np.linalg.norm(bn[r])
