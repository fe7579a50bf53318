"""GPU parity of the scalar SIPG apply (C ABI, FP64 and FP32) against the CPU oracle.

Error metric: max_i |y_i - y_ref,i| / max_i |y_ref,i|. FP64 must agree to 1e-12, FP32
(storage and accumulation) to 1e-5, on identical seeded inputs. Small cases span several
thread blocks with a ragged last block; the full 64^3 trilinear configuration is checked
on sampled cells that the oracle evaluates one by one.
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
TOL32 = 1e-5


def relerr(y, ref):
    return float(np.abs(y - ref).max() / np.abs(ref).max())


def run_case(n, k, geom="affine", theta=-1.0, c=1.0, mask=0b111111, pen_mode=0, alpha=2.0, kappa=False,
             precision=dg.DG_FP64, nrhs=1, seed=0):
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    mesh = dg.Mesh(*n, verts)
    op = dg.Operator(mesh, k, c=c, theta=theta, dirichlet_mask=mask, penalty_mode=pen_mode, penalty_alpha=alpha,
                     precision=precision, max_rhs=nrhs)
    ncell = mesh.ncell
    orc = oracle.Problem(*n, k, vertices=verts, c=c, theta=theta, dirichlet_mask=mask, pen_mode=pen_mode,
                         pen_alpha=alpha)
    if kappa:
        kv, kf = wl.lognormal_kappa(ncell, k + 1, seed=2)
        orc.kappa_vol, orc.kappa_face = kv, kf
        tkv = torch.from_numpy(kv).to("cuda", op.dtype)
        tkf = torch.from_numpy(kf).to("cuda", op.dtype)
        op.set_kappa(tkv, tkf)
    xs = np.stack([wl.uniform_vector(op.ndofs, seed + r) for r in range(nrhs)])
    xd = torch.from_numpy(xs).to("cuda", op.dtype)
    y = op.apply(xd if nrhs > 1 else xd[0]).double().cpu().numpy().reshape(nrhs, -1)
    torch.cuda.synchronize()
    refs = np.stack([orc.apply(xs[r]) for r in range(nrhs)])
    return max(relerr(y[r], refs[r]) for r in range(nrhs))


# config 1: 4^3 affine cells, Q2, c = 1, SIPG, penalty 2k(k+1)/h, Dirichlet, x ~ U[-1,1] seed 0
def test_config1_affine_q2_fp64():
    assert run_case((4, 4, 4), 2) <= TOL64


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_degrees_ragged_mesh_fp64(k, geom):
    # 5 x 3 x 4 cells: several blocks per launch and a ragged last block for every degree
    assert run_case((5, 3, 4), k, geom) <= TOL64


@pytest.mark.parametrize("theta,mask,pen_mode,c", [(1.0, 0b101101, 0, 0.5), (0.0, 0b010110, 1, 0.0),
                                                   (-1.0, 0, 1, 2.0)])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_theta_masks_penalty_modes(theta, mask, pen_mode, c, geom):
    assert run_case((3, 4, 2), 2, geom, theta=theta, c=c, mask=mask, pen_mode=pen_mode, alpha=3.0) <= TOL64


@pytest.mark.parametrize("geom", ["affine", "trilinear"])
@pytest.mark.parametrize("k", [2, 3])
def test_pointwise_kappa(geom, k):
    assert run_case((4, 3, 3), k, geom, kappa=True) <= TOL64


def test_single_cell_and_thin_meshes():
    assert run_case((1, 1, 1), 3, "trilinear") <= TOL64
    assert run_case((7, 1, 1), 2) <= TOL64
    assert run_case((1, 2, 9), 4, "trilinear") <= TOL64


def test_multiple_rhs_fp64():
    assert run_case((3, 3, 4), 3, "trilinear", nrhs=5) <= TOL64


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
def test_fp32_against_fp64_oracle(k, geom):
    err = run_case((4, 3, 5), k, geom, precision=dg.DG_FP32, nrhs=2)
    print(f"FP32 Q{k} {geom}: rel err {err:.2e}")
    assert err <= TOL32


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("kappa", [False, True])
def test_fp32_recomputed_geometry(k, kappa):
    """FP32 on a trilinear mesh with the geometry recomputed in the kernels (nothing
    stored): forward apply and transposed apply against the FP64 oracle."""
    n = (4, 3, 5)
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), k, precision=dg.DG_FP32, geometry=dg.DG_GEOM_RECOMPUTE, max_rhs=2,
                     theta=1.0)
    assert op.stats().geometry == dg.DG_GEOM_RECOMPUTE
    orc = oracle.Problem(*n, k, vertices=verts, theta=1.0)
    if kappa:
        kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
        orc.kappa_vol, orc.kappa_face = kv, kf
        op.set_kappa(torch.from_numpy(kv).float().cuda(), torch.from_numpy(kf).float().cuda())
    xs = np.stack([wl.uniform_vector(op.ndofs, 20 + r) for r in range(2)])
    xd = torch.from_numpy(xs).float().cuda()
    y = op.apply(xd).double().cpu().numpy()
    yt = torch.empty_like(xd)
    dg.dg_apply_adjoint(op.handle, xd.data_ptr(), None, yt.data_ptr(), None, None, None, nrhs=2)
    yt = yt.double().cpu().numpy()
    for r in range(2):
        assert relerr(y[r], orc.apply(xs[r])) <= TOL32
        assert relerr(yt[r], orc.apply(xs[r], transpose=True)) <= TOL32


@pytest.mark.parametrize("case", ["fp64_q3_2rhs", "fp64_4cells", "fp64_kappa_3rhs", "fp32_three_kernel",
                                  "df64_q3", "fp32_fused_unpipelined"])
def test_apply_host_matches_device(case):
    # dg_apply_host runs the three-kernel apply in chunks of cells with the copies overlapped
    # (one chunk per cell when there are fewer cells than chunks); other variants copy, apply
    # and copy back. Either way the result is the device apply's, bit for bit.
    cfg = {"fp64_q3_2rhs": ((4, 4, 3), 3, dg.DG_FP64, 2, True, False, None),
           "fp64_4cells": ((2, 2, 1), 2, dg.DG_FP64, 1, True, False, None),
           "fp64_kappa_3rhs": ((9, 7, 5), 2, dg.DG_FP64, 3, True, True, None),
           "fp32_three_kernel": ((7, 6, 5), 2, dg.DG_FP32, 3, True, False, None),
           "df64_q3": ((6, 5, 4), 3, dg.DG_FP64, 2, True, False, dg.DG_VARIANT_DF64),
           "fp32_fused_unpipelined": ((6, 5, 4), 3, dg.DG_FP32, 2, False, False, dg.DG_VARIANT_FUSED)}[case]
    n, k, prec, nrhs, curved, kappa, variant = cfg
    verts = wl.perturbed_vertices(*n, seed=1) if curved else None
    op = dg.Operator(dg.Mesh(*n, verts), k, precision=prec, max_rhs=nrhs)
    if kappa:
        kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
        op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    if variant is not None:
        op.set_variant(variant)
    dt = np.float64 if prec == dg.DG_FP64 else np.float32
    x = np.stack([wl.uniform_vector(op.ndofs, s) for s in range(nrhs)]).astype(dt)
    xh, yh = torch.from_numpy(x).pin_memory(), torch.zeros(x.shape, dtype=torch.from_numpy(x).dtype).pin_memory()
    op.apply_host(xh if nrhs > 1 else xh[0], yh if nrhs > 1 else yh[0])
    yd = op.apply(torch.from_numpy(x).cuda() if nrhs > 1 else torch.from_numpy(x[0]).cuda()).cpu().numpy()
    assert np.array_equal(yh.numpy().reshape(yd.shape), yd)


def test_apply_is_deterministic():
    n, k = (6, 5, 4), 4
    op = dg.Operator(dg.Mesh(*n, wl.perturbed_vertices(*n, seed=1)), k)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).cuda()
    y1 = op.apply(x)
    y2 = op.apply(x)
    assert torch.equal(y1, y2)


def test_argument_errors_on_device():
    op = dg.Operator(dg.Mesh(2, 2, 2), 2, max_rhs=2)
    x = torch.zeros(op.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError):
        dg.dg_apply(op.handle, x.data_ptr(), x.data_ptr(), 1, None)  # aliased
    with pytest.raises(dg.DGError):
        dg.dg_apply(op.handle, x.data_ptr(), x.data_ptr() + 8, 1, None)  # misaligned
    with pytest.raises(dg.DGError):
        dg.dg_apply(op.handle, x.data_ptr(), 0, 1, None)
    y = torch.empty(3 * op.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError):
        dg.dg_apply(op.handle, y.data_ptr(), y[op.ndofs:].data_ptr(), 3, None)  # nrhs > max_rhs
    with pytest.raises(TypeError):
        op.apply(x.float())


# config 2 at full size: 64^3 trilinear-perturbed cells, FP64, sampled cells vs the oracle
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_config2_full_size_sampled(k):
    n = (64, 64, 64)
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), k)
    x = wl.uniform_vector(op.ndofs, 0)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy().reshape(op.mesh.ncell, -1)
    cells = wl.sample_cells(op.mesh.ncell, 96, seed=7 + k)
    orc = oracle.Problem(*n, k, vertices=verts)
    ref = orc.apply_cells(x, cells, nthreads=0)
    err = float(np.abs(y[cells] - ref).max() / np.abs(ref).max())
    assert err <= TOL64, err


def test_config2_q3_tuned_as_benchmarked_sampled():
    """The operator exactly as the benchmark times it: 64^3 trilinear Q3, FP64, blocking
    chosen by dg_operator_autotune, and then the same operator in double-float with its
    own tuned blocking; sampled cells against the oracle."""
    n, k = (64, 64, 64), 3
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), k)
    op.autotune(1)
    x = wl.uniform_vector(op.ndofs, 0)
    xd = torch.from_numpy(x).cuda()
    cells = wl.sample_cells(op.mesh.ncell, 96, seed=31)
    ref = oracle.Problem(*n, k, vertices=verts).apply_cells(x, cells, nthreads=0)
    y = op.apply(xd).cpu().numpy().reshape(op.mesh.ncell, -1)
    assert float(np.abs(y[cells] - ref).max() / np.abs(ref).max()) <= TOL64
    op.set_variant(dg.DG_VARIANT_DF64)
    op.autotune(1)
    y = op.apply(xd).cpu().numpy().reshape(op.mesh.ncell, -1)
    assert float(np.abs(y[cells] - ref).max() / np.abs(ref).max()) <= TOL64


# ---------------------------------------------------------------- fused persistent variant

def run_fused(n, k, precision, nrhs=1, tile=0, theta=-1.0, mask=0b111111, c=1.0):
    op = dg.Operator(dg.Mesh(*n), k, precision=precision, max_rhs=nrhs, theta=theta, dirichlet_mask=mask, c=c)
    op.set_variant(dg.DG_VARIANT_FUSED, tile)
    assert op.stats().variant == dg.DG_VARIANT_FUSED
    orc = oracle.Problem(*n, k, theta=theta, dirichlet_mask=mask, c=c)
    xs = np.stack([wl.uniform_vector(op.ndofs, r) for r in range(nrhs)])
    y = op.apply(torch.from_numpy(xs).to("cuda", op.dtype)).double().cpu().numpy()
    assert op.stats().persistent_grid > 0
    return max(relerr(y[r], orc.apply(xs[r])) for r in range(nrhs))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_fused_fp64_matches_oracle(k):
    # rows of 8/4/2 cells along x: 11 cells leave a ragged last tile
    assert run_fused((11, 3, 4), k, dg.DG_FP64) <= TOL64


@pytest.mark.parametrize("tile", [1, 3, 16])
def test_fused_tiles_theta_masks_and_rhs(tile):
    assert run_fused((5, 4, 3), 2, dg.DG_FP64, nrhs=3, tile=tile, theta=1.0, mask=0b100111, c=0.5) <= TOL64


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_fused_fp32(k):
    err = run_fused((9, 4, 5), k, dg.DG_FP32, nrhs=4)
    print(f"fused FP32 Q{k}: rel err {err:.2e}")
    assert err <= TOL32


def test_fused_is_the_fp32_affine_default_and_rejected_elsewhere():
    assert dg.Operator(dg.Mesh(3, 3, 3), 3, precision=dg.DG_FP32).stats().variant == dg.DG_VARIANT_FUSED
    assert dg.Operator(dg.Mesh(3, 3, 3), 2, precision=dg.DG_FP32).stats().variant == dg.DG_VARIANT_CELLWISE
    assert dg.Operator(dg.Mesh(3, 3, 3), 2).stats().variant == dg.DG_VARIANT_THREE_KERNEL
    op = dg.Operator(dg.Mesh(3, 3, 3, wl.perturbed_vertices(3, 3, 3)), 2, precision=dg.DG_FP32)
    assert op.stats().variant == dg.DG_VARIANT_THREE_KERNEL
    with pytest.raises(dg.DGError) as e:
        op.set_variant(dg.DG_VARIANT_FUSED)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED


# ---------------------------------------------------------------- cellwise persistent variant

def run_cellwise(n, k, precision, nrhs=1, brick=0, theta=-1.0, mask=0b111111, c=1.0):
    op = dg.Operator(dg.Mesh(*n), k, precision=precision, max_rhs=nrhs, theta=theta, dirichlet_mask=mask, c=c)
    op.set_variant(dg.DG_VARIANT_CELLWISE, brick)
    st = op.stats()
    assert st.variant == dg.DG_VARIANT_CELLWISE and st.cells_per_block == (brick or (256 if precision == dg.DG_FP32 and k == 2 else 128))
    orc = oracle.Problem(*n, k, theta=theta, dirichlet_mask=mask, c=c)
    xs = np.stack([wl.uniform_vector(op.ndofs, r) for r in range(nrhs)])
    y = op.apply(torch.from_numpy(xs).to("cuda", op.dtype)).double().cpu().numpy()
    assert op.stats().persistent_grid > 0
    return max(relerr(y[r], orc.apply(xs[r])) for r in range(nrhs))


@pytest.mark.parametrize("k,brick", [(1, 64), (1, 128), (1, 256), (2, 64), (2, 128), (2, 256)])
def test_cellwise_fp64_matches_oracle(k, brick):
    # bricks of 8 x 4 x (brick/32) cells: 19 x 6 x 11 cells leave ragged bricks on all axes
    # and brick-boundary faces in every direction
    assert run_cellwise((19, 6, 11), k, dg.DG_FP64, brick=brick) <= TOL64


@pytest.mark.parametrize("n", [(1, 1, 1), (3, 2, 2), (8, 4, 2), (17, 9, 3), (2, 13, 20)])
def test_cellwise_meshes_smaller_and_larger_than_a_brick(n):
    assert run_cellwise(n, 2, dg.DG_FP64, brick=64) <= TOL64


@pytest.mark.parametrize("mask,theta,c", [(0b100111, 1.0, 0.5), (0, -1.0, 0.0), (0b010101, 0.0, 2.0)])
def test_cellwise_theta_masks_and_rhs(mask, theta, c):
    assert run_cellwise((10, 5, 9), 2, dg.DG_FP64, nrhs=3, brick=64, theta=theta, mask=mask, c=c) <= TOL64


@pytest.mark.parametrize("k", [1, 2])
def test_cellwise_fp32(k):
    err = run_cellwise((19, 6, 11), k, dg.DG_FP32, nrhs=4, brick=128)
    print(f"cellwise FP32 Q{k}: rel err {err:.2e}")
    assert err <= TOL32


def test_cellwise_rejected_where_it_does_not_apply():
    for op in (dg.Operator(dg.Mesh(3, 3, 3), 3, precision=dg.DG_FP32),
               dg.Operator(dg.Mesh(3, 3, 3, wl.perturbed_vertices(3, 3, 3)), 2, precision=dg.DG_FP32)):
        with pytest.raises(dg.DGError) as e:
            op.set_variant(dg.DG_VARIANT_CELLWISE)
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
    op = dg.Operator(dg.Mesh(3, 3, 3), 2, precision=dg.DG_FP32)
    for bad in (32, 96, 512):
        with pytest.raises(dg.DGError):
            op.set_variant(dg.DG_VARIANT_CELLWISE, bad)


@pytest.mark.parametrize("brick", [64, 256])
def test_cellwise_fp32_bricks_and_rhs(brick):
    assert run_cellwise((21, 7, 17), 2, dg.DG_FP32, nrhs=3, brick=brick, theta=1.0, mask=0b011110) <= TOL32


@pytest.mark.parametrize("n,brick,nrhs", [((16, 8, 16), 256, 2), ((20, 9, 17), 256, 3), ((24, 13, 10), 128, 2),
                                          ((12, 6, 5), 64, 2), ((8, 4, 8), 256, 1), ((36, 18, 34), 256, 4)])
def test_cellwise_fp32_bulk_staged(n, brick, nrhs):
    # nx a multiple of 4: whole bricks take their x rows and brick-boundary neighbours into
    # shared memory by bulk copies one item ahead, ragged bricks by loads. In the largest
    # case (500 items, more than one wave of blocks) blocks run several items, mixing both.
    assert dg.dg_device_faults(clear=True) == 0
    assert run_cellwise(n, 2, dg.DG_FP32, nrhs=nrhs, brick=brick) <= TOL32
    assert dg.dg_device_faults() == 0


def test_config4_fp64_full_size_sampled():
    # the FP64 operator of config 4 (128^3 affine cells, Q2): residuals of the refinement
    # and the all-FP64 CG; 16 right-hand sides through the tuned three-kernel apply
    n, k, nrhs = (128, 128, 128), 2, 16
    op = dg.Operator(dg.Mesh(*n), k, max_rhs=nrhs)
    b = wl.refinement_rhs(*n, 27, seeds=range(nrhs))
    y = op.apply(torch.from_numpy(b).cuda()).cpu().numpy().reshape(nrhs, op.mesh.ncell, 27)
    cells = wl.sample_cells(op.mesh.ncell, 48, seed=18)
    orc = oracle.Problem(*n, k)
    for r in (0, 9, 15):
        ref = orc.apply_cells(b[r], cells)
        assert float(np.abs(y[r][cells] - ref).max() / np.abs(ref).max()) <= TOL64


def test_config4_fp32_16rhs_full_size_sampled():
    # 128^3 affine cells, Q2, FP32, 16 right-hand sides in one persistent launch
    n, k, nrhs = (128, 128, 128), 2, 16
    op = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32, max_rhs=nrhs)
    b = wl.refinement_rhs(*n, 27, seeds=range(nrhs), dtype=np.float32)
    y = op.apply(torch.from_numpy(b).cuda()).cpu().numpy().reshape(nrhs, op.mesh.ncell, 27)
    cells = wl.sample_cells(op.mesh.ncell, 48, seed=17)
    orc = oracle.Problem(*n, k)
    for r in (0, 7, 15):
        ref = orc.apply_cells(b[r].astype(np.float64), cells)
        assert float(np.abs(y[r][cells] - ref).max() / np.abs(ref).max()) <= TOL32


@pytest.mark.parametrize("precision,geom", [(dg.DG_FP64, "trilinear"), (dg.DG_FP32, "affine")])
def test_autotune_keeps_parity(precision, geom):
    n, k = (6, 5, 7), 3
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    op = dg.Operator(dg.Mesh(*n, verts), k, precision=precision, max_rhs=2)
    res = op.autotune(nrhs=2)
    assert res["candidates"] > 3 and res["ms_best"] > 0 and res["ms_best"] <= res["ms_default"] * 1.5
    st = op.stats()
    assert st.variant == res["variant"]
    xs = np.stack([wl.uniform_vector(op.ndofs, r) for r in range(2)])
    y = op.apply(torch.from_numpy(xs).to("cuda", op.dtype)).double().cpu().numpy()
    orc = oracle.Problem(*n, k, vertices=verts)
    tol = TOL64 if precision == dg.DG_FP64 else TOL32
    for r in range(2):
        assert relerr(y[r], orc.apply(xs[r])) <= tol


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("geom", ["affine", "trilinear"])
@pytest.mark.parametrize("arith", ["fp64", "fp32", "df64"])
def test_overintegration_k_plus_2_points(k, geom, arith):
    # m = k + 2 Gauss points: the point kernels (FP64) and the line kernels (FP32,
    # double-float) with M = P + 1
    n = (4, 3, 5)
    verts = wl.perturbed_vertices(*n, seed=1) if geom == "trilinear" else None
    m = k + 2
    op = dg.Operator(dg.Mesh(*n, verts), k, quad_points=m,
                     precision=dg.DG_FP32 if arith == "fp32" else dg.DG_FP64)
    orc = oracle.Problem(*n, k, m=m, vertices=verts)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, m, seed=2)
    op.set_kappa(torch.from_numpy(kv).to("cuda", op.dtype), torch.from_numpy(kf).to("cuda", op.dtype))
    if arith == "df64":
        op.set_variant(dg.DG_VARIANT_DF64)
    orc.kappa_vol, orc.kappa_face = kv, kf
    x = wl.uniform_vector(op.ndofs, 0)
    y = op.apply(torch.from_numpy(x).to("cuda", op.dtype)).double().cpu().numpy()
    assert relerr(y, orc.apply(x)) <= (TOL32 if arith == "fp32" else TOL64)
    with pytest.raises(dg.DGError):
        op.set_variant(dg.DG_VARIANT_FUSED)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_recomputed_geometry_forward(k):
    # DG_GEOM_RECOMPUTE: no stored per-point geometry; the apply recomputes it from the vertices
    n = (4, 3, 5)
    verts = wl.perturbed_vertices(*n, seed=1)
    op = dg.Operator(dg.Mesh(*n, verts), k, theta=1.0, max_rhs=2, geometry=dg.DG_GEOM_RECOMPUTE)
    assert op.stats().geometry == dg.DG_GEOM_RECOMPUTE
    orc = oracle.Problem(*n, k, vertices=verts, theta=1.0)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    op.set_kappa(torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda())
    orc.kappa_vol, orc.kappa_face = kv, kf
    xs = np.stack([wl.uniform_vector(op.ndofs, r) for r in range(2)])
    y = op.apply(torch.from_numpy(xs).cuda()).cpu().numpy()
    for r in range(2):
        assert relerr(y[r], orc.apply(xs[r])) <= TOL64
    with pytest.raises(dg.DGError) as e:  # over-integration needs stored geometry
        dg.Operator(dg.Mesh(*n, verts), k, quad_points=k + 2, geometry=dg.DG_GEOM_RECOMPUTE)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
