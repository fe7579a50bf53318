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
@pytest.mark.parametrize("n", [(5, 4, 3), (5, 3, 3)])
def test_block_jacobi_fp32(k, n):
    # (5, 3, 3) at k = 2: 1215 values per right-hand side, not a multiple of 4 (no 16-byte rows)
    err = run(n, k, precision=dg.DG_FP32, nrhs=3, per_cell=True)
    print(f"block Jacobi FP32 Q{k} {n}: rel err {err:.2e}")
    assert err <= TOL32


def test_block_jacobi_fp32_many_chunks():
    # one thread per cell over 381 chunks of 128 cells (the last one ragged), 16-byte rows
    n, k, nrhs = (41, 36, 33), 2, 2
    op = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32, max_rhs=nrhs)
    rs = np.stack([wl.uniform_vector(op.ndofs, s) for s in (4, 5)])
    z = op.block_jacobi(torch.from_numpy(rs).float().cuda()).double().cpu().numpy().reshape(nrhs, op.mesh.ncell, 27)
    rn = rs.astype(np.float32).astype(np.float64).reshape(nrhs, op.mesh.ncell, 27)
    orc = oracle.Problem(*n, k)
    for cell in list(wl.sample_cells(op.mesh.ncell, 24, seed=6)) + [op.mesh.ncell - 1]:
        for i in range(nrhs):
            zc = np.zeros(op.ndofs)
            zc[cell * 27:(cell + 1) * 27] = z[i, cell]
            Az = orc.apply_cells(zc, np.array([cell]))[0]
            assert np.abs(Az - rn[i, cell]).max() <= TOL32 * np.abs(rn[i, cell]).max()


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


def pcg_steps(A, precond, b, m):
    """m steps of preconditioned CG from x = 0 in FP64 (the textbook recursion)."""
    x, r = np.zeros_like(b), b.copy()
    z = precond(r)
    p, rz = z.copy(), r @ z
    for _ in range(m):
        Ap = A @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


@pytest.mark.parametrize("n,k", [((6, 5, 7), 2), ((8, 4, 6), 2), ((9, 5, 4), 1)])
def test_fp32_block_jacobi_cg_steps_match_fp64_recursion(n, k):
    # The FP32 CG applies the cell-block inverse inside its two vector passes (r -= alpha Ap
    # with z = B r and the r.z, r.r partials; then x += alpha p, p = B r + beta p). After m
    # iterations its x must be the FP64 recursion's x up to FP32 rounding: a wrong alpha,
    # beta, x or p update would be off by O(1). (6, 5, 7): rows not a multiple of 4 values;
    # (8, 4, 6): one full and one ragged chunk of 128 cells.
    nrhs, m = 3, 6
    op = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32, max_rhs=nrhs)
    orc = oracle.Problem(*n, k)
    A = orc.assemble()
    bn = wl.refinement_rhs(*n, (k + 1) ** 3, seeds=range(nrhs)).astype(np.float32)
    b = torch.from_numpy(bn).cuda()
    x = torch.zeros_like(b)
    opt = dg.dg_cg_options(1e-14, m, 1, 1, dg.DG_PRECOND_BLOCK_JACOBI)
    ok, info = dg.dg_cg_solve(op.handle, b.data_ptr(), x.data_ptr(), nrhs, opt, None)
    assert not ok and all(i["iters"] == m for i in info)
    for r in range(nrhs):
        ref = pcg_steps(A, orc.block_jacobi, bn[r].astype(np.float64), m)
        err = relerr(x[r].double().cpu().numpy(), ref)
        print(f"FP32 block-Jacobi CG, {m} steps, Q{k} {n}: rel err vs FP64 recursion {err:.2e}")
        assert err <= 1e-4
