#!/usr/bin/env python3
"""Throughput of the matrix-free SIPG-DG apply y = A x on one GB300 (or N replicas).

Workload (one "step"): one FP64 apply of the scalar diffusion-reaction SIPG operator,
c = 1, penalty 2k(k+1)/h, on 64^3 cells whose interior vertices are perturbed by up to
0.1h (seed 1), per-quadrature-point geometry, degree Q3 with 4^3 Gauss points (16.8M
DOFs), x ~ U[-1,1] (seed 0): the volume kernel, the interior and boundary face kernel
and the back-projection kernel. Every input (x 134 MB, geometry 1.6 GB) is larger than
the 129 MB L2, so no flush is needed between steps.

Besides the headline the line carries (rank 0, one GPU): the Q1-Q5 sweep in FP64,
double-float and FP32 (each FP32 result's error against the FP64 apply of the same x),
config 4's FP32 apply of 16 right-hand sides, Stokes, the adjoint, and config 4's solve
to 1e-10 (128^3, Q2, 16 right-hand sides): mixed CG with reliable updates and FP64
refinement around FP32 CG against the all-FP64 CG with and without block Jacobi. Every
roofline fraction is max(F / peak, B_alg / HBM) over the measured time, F the executed
flops and B_alg the algorithm's own bytes (x, y, vertex coordinates).

Prints one JSON line (rank 0). With --gpus N > 1 (torchrun) every rank applies its own
replica of the workload (no collective on the data path) and value = total DOF/s.
``--impl reference`` times the CPU oracle instead (the only baseline that exists for
this method), on the host cores, with bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1812_08075_gb300 import workloads as wl  # noqa: E402

METRIC = "dg_apply DOF/s (FP64 and mixed) at Q2-Q5; % of FP64-peak / HBM roofline"
N_CELLS = 64
VARIANT_NAMES = {1: "three-kernel", 2: "fused persistent", 3: "cellwise persistent", 4: "double-float three-kernel"}
PRECOND_NAMES = {0: "none", 1: "point Jacobi (diagonal set up outside the timed solves)",
                 2: "cell-block Jacobi by fast diagonalisation (set up outside the timed solves)"}
FP64_FLOPS_PER_SM_CLK = 4.0   # 2 DFMA per SM per clock: 1.25 TFLOP/s nominal at 2.07 GHz
FP32_FLOPS_PER_SM_CLK = 256.0  # 128 FFMA per SM per clock
# DRAM bytes (read + write) per cell of one k_cell launch, from an ncu capture of the
# 40^3 Q3 case (262.4 MB + 103.9 MB for 64000 cells); the kernel's traffic is
# proportional to the number of cells, so it scales to a full launch by cells.
KCELL_Q3_DRAM_BYTES_PER_CELL = (262.393344e6 + 103.932928e6) / 40 ** 3


def sm_count() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def peaks(probe: bool = False):
    """Roofline denominators: HBM from the driver's measured copy bandwidth; FP64 and FP32
    derived from the pipes' per-clock rates, the device's SM count and the maximum SM
    clock; with probe, also the FMA throughput this run measures (dg_measure_fma_peak)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mp = json.load(open(path)) if os.path.exists(path) else {}
    clk = float(mp.get("sm_max_mhz", 2070.0)) * 1e6
    sms = sm_count()
    out = {
        "hbm_gbs": float(mp.get("hbm_gbs", 6800.0)),
        "hbm_src": "measured" if "hbm_gbs" in mp else "fallback",
        "fp64_tflops": sms * FP64_FLOPS_PER_SM_CLK * clk / 1e12,
        "fp32_tflops": sms * FP32_FLOPS_PER_SM_CLK * clk / 1e12,
        "clk_mhz": clk / 1e6,
        "sms": sms,
    }
    if probe:
        from paper_1812_08075_gb300 import dg
        out["fp64_probe_tflops"] = dg.dg_measure_fma_peak(dg.DG_FP64)
        out["fp32_probe_tflops"] = dg.dg_measure_fma_peak(dg.DG_FP32)
    return out


def roofline_entry(flops, alg_bytes, ms, pk, fp32, impl_bytes=None):
    """Fraction of the roofline time max(F / peak, B_alg / HBM) over the measured time:
    F = the executed kernels' exact flop count (equal to ncu's FP instruction count and
    below the analytic model of the algorithm), B_alg = x read + y written (+ vertex
    coordinates, + kappa), the algorithm's own bytes; stored geometry and scratch are
    implementation bytes, reported apart."""
    peak = pk["fp32_tflops"] if fp32 else pk["fp64_tflops"]
    t_alu = flops / (peak * 1e12)
    t_mem = alg_bytes / (pk["hbm_gbs"] * 1e9)
    t = ms * 1e-3
    out = {"bound": "alu" if t_alu >= t_mem else "hbm", "roofline_frac": max(t_alu, t_mem) / t,
           "tflops": flops / t / 1e12, "frac_alu_peak": flops / t / 1e12 / peak,
           "alg_bytes": alg_bytes, "alg_gbs": alg_bytes / t / 1e9, "frac_hbm_alg": alg_bytes / t / 1e9 / pk["hbm_gbs"],
           "flops": flops}
    if impl_bytes is not None:
        out["impl_bytes_model"] = impl_bytes
    return out


def workload_config(k: int):
    l2 = ("inputs larger than L2 (x 134 MB, stored geometry 1.6 GB at Q3), no flush" if N_CELLS >= 64
          else "smaller profiling case")
    return {"workload": f"scalar SIPG diffusion-reaction, {N_CELLS}^3 trilinear-perturbed cells (0.1h, seed 1), "
                        f"Q{k}, {k + 1}^3 Gauss points, c=1, penalty 2k(k+1)/h, Dirichlet, FP64 apply",
            "cells": N_CELLS ** 3, "degree": k, "ndofs": N_CELLS ** 3 * (k + 1) ** 3,
            "l2": l2,
            "parallelism": "replicas (independent problem per GPU)"}


# ------------------------------------------------------------------- clocks sampling

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts, float(parts[2]), float(parts[3]), parts[4], parts[6:10]))
            except (ValueError, IndexError):
                continue
        os.unlink(self.f.name)
        timed = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        window = "timed region"
        if len(timed) < 3:
            timed, window = rows, "warm-up and timed region"
        if not timed:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in timed for i, v in enumerate(r[4]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[1] for r in timed), "sm_max_mhz": max(r[2] for r in timed),
                "reasons": reasons, "samples": len(timed), "window": window,
                "power_w_max": max((float(r[3]) for r in timed if r[3] not in ("[N/A]", "N/A")), default=None)}


# ------------------------------------------------------------------- CPU oracle timing

def oracle_rate(k: int, target_core_seconds: float, cores: int, seed: int = 11):
    """DOF/s of the oracle's cell-gather apply on a bounded random sample of cells."""
    import oracle
    n = (N_CELLS,) * 3
    verts = wl.perturbed_vertices(*n, seed=1)
    prob = oracle.Problem(*n, k, vertices=verts)
    x = wl.uniform_vector(prob.ncell * (k + 1) ** 3, 0)
    probe = wl.sample_cells(prob.ncell, 512, seed=seed)
    t = time.perf_counter()
    prob.apply_cells(x, probe, nthreads=cores)
    dt = max(time.perf_counter() - t, 1e-6)
    per_cell_core_s = dt * cores / probe.size
    ncells = int(min(prob.ncell, max(512, target_core_seconds / per_cell_core_s)))
    cells = wl.sample_cells(prob.ncell, ncells, seed=seed + 1)
    t = time.perf_counter()
    prob.apply_cells(x, cells, nthreads=cores)
    dt = time.perf_counter() - t
    return cells.size * (k + 1) ** 3 / dt, cells.size, dt


def host_cores():
    return len(os.sched_getaffinity(0))


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = host_cores()
    k = args.degree
    n = (N_CELLS,) * 3
    verts = wl.perturbed_vertices(*n, seed=1)
    prob = oracle.Problem(*n, k, vertices=verts)
    x = wl.uniform_vector(prob.ncell * (k + 1) ** 3, 0)
    # size one step to about 1 s of wall time on the host cores
    probe = wl.sample_cells(prob.ncell, 512, seed=21)
    t = time.perf_counter()
    prob.apply_cells(x, probe, nthreads=cores)
    per_cell = (time.perf_counter() - t) / probe.size
    ncells = int(min(prob.ncell, max(256, 1.0 / per_cell)))
    samples = [wl.sample_cells(prob.ncell, ncells, seed=100 + s) for s in range(args.warmup + args.steps)]
    for s in samples[:args.warmup]:
        prob.apply_cells(x, s, nthreads=cores)
    t = time.perf_counter()
    dofs = 0
    for s in samples[args.warmup:]:
        prob.apply_cells(x, s, nthreads=cores)
        dofs += s.size * (k + 1) ** 3
    dt = time.perf_counter() - t
    value = dofs / dt
    sample = (f"{ncells} random cells per step of the {N_CELLS}^3 Q{k} workload (cell-gather form: each cell's "
              f"volume term and its six faces), {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(k),
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------- GPU path

def aggregate(ms_local: float, ndofs: int, world: int, dist, device="cuda"):
    """Whole-job result of a replica run: the slowest rank's milliseconds per step (max
    over ranks) and value = total DOFs of all ranks / that time."""
    ms = ms_local
    if dist is not None:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * ndofs / (ms * 1e-3)


def time_applies(op, x, y, steps, warmup, dist, profile=False):
    import torch
    from paper_1812_08075_gb300 import dg
    for _ in range(warmup):
        op.apply(x, y)
    if profile:
        dg.dg_operator_profile(op.handle, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        op.apply(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / steps
    kt = None
    if profile:
        kms, napp = dg.dg_operator_kernel_times(op.handle)
        dg.dg_operator_profile(op.handle, False)
        kt = [v / max(napp, 1) for v in kms]
    return ms, kt, (t0, t1)


def config4_rhs(op64, n, k, nrhs):
    """Config 4's right-hand sides b_s = l / max|l| + eta_s (seeds 0..nrhs-1) on the device:
    l_i = (sin pi x sin pi y sin pi z, phi_i), the source evaluated at the library's own
    Gauss points and integrated by its data-term kernel (dg_rhs)."""
    import torch
    from paper_1812_08075_gb300 import dg
    nodes = dg.dg_reference_tables(k)["gauss_nodes"]
    f = torch.from_numpy(wl.sin_product_source(n, n, n, nodes)).cuda()
    l = op64.rhs(f)
    del f
    l = l / l.abs().max()
    b = torch.empty(nrhs, op64.ndofs, dtype=torch.float64, device="cuda")
    for s in range(nrhs):
        b[s] = l + torch.from_numpy(wl.uniform_vector(op64.ndofs, s)).cuda()
    torch.cuda.synchronize()
    return b


def mixed_apply(pk, n_cells=128, k=2, nrhs=16):
    """Config 4's operator (affine 128^3, Q2): the FP32 apply of 16 right-hand sides in one
    persistent launch, next to the FP64 apply of the same 16 vectors, with the FP32
    result's error against the FP64 one."""
    import torch
    from paper_1812_08075_gb300 import dg
    mesh = dg.Mesh(n_cells, n_cells, n_cells)
    res = {"workload": f"scalar SIPG, {n_cells}^3 affine cells, Q{k}, {nrhs} right-hand sides "
                       f"(Gauss-projected sin-product load vector + U[-1,1] noise, seeds 0-{nrhs - 1})"}
    ys = {}
    b = None
    for prec, tag in ((dg.DG_FP64, "fp64"), (dg.DG_FP32, "fp32")):
        op = dg.Operator(mesh, k, precision=prec, max_rhs=nrhs)
        if b is None:
            b = config4_rhs(op, n_cells, k, nrhs)
        res.setdefault("tuning", {})[tag] = op.autotune(nrhs)
        xx = b.to(op.dtype)
        yy = torch.empty_like(xx)
        ms, kt, _ = time_applies(op, xx, yy, 10, 3, None, profile=True)
        st = op.stats()
        f = sum(st.flops) * nrhs
        alg = st.dofs_bytes * nrhs  # x read + y written, affine mesh (no vertices)
        ent = {"dof_s": nrhs * op.ndofs / (ms * 1e-3), "ms_per_apply": ms, "variant": VARIANT_NAMES[st.variant],
               "persistent_grid": st.persistent_grid, "kernel_ms": kt}
        ent.update(roofline_entry(f, alg, ms, pk, prec == dg.DG_FP32, impl_bytes=sum(st.bytes) * nrhs))
        if prec == dg.DG_FP64:
            ys["fp64"] = yy
        else:
            y64 = ys["fp64"]
            err = [float((yy[s].double() - y64[s]).abs().max() / y64[s].abs().max()) for s in range(nrhs)]
            ent["err_vs_fp64"] = max(err)
            ent["err_note"] = "max over right-hand sides of max|y32 - y64| / max|y64| (y64: the FP64 apply above)"
        res[tag] = ent
        del op, xx
        if prec == dg.DG_FP32:
            del yy
    del ys, b
    return res


def stokes_apply(pk, n_cells=32, k=3):
    """Config 3: DG Stokes block operator, 32^3 affine cells, velocity Q3 / pressure Q2."""
    import torch
    from paper_1812_08075_gb300 import dg
    op = dg.Operator(dg.Mesh(n_cells, n_cells, n_cells), k, problem=dg.DG_STOKES, dirichlet_mask=0b111101)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).cuda()
    y = torch.empty_like(x)
    ms, kt, _ = time_applies(op, x, y, 20, 3, None, profile=True)
    f = sum(op.stats().flops)
    # the same operator in double-float arithmetic (DG_VARIANT_DF64), blockings tuned
    y64 = y.clone()
    op.set_variant(dg.DG_VARIANT_DF64)
    op.autotune(1)
    ms_d, kt_d, _ = time_applies(op, x, y, 20, 3, None, profile=True)
    df = {"dof_s": op.ndofs / (ms_d * 1e-3), "ms": ms_d, "kernel_ms": kt_d, "speedup_over_fp64": ms / ms_d,
          "fp64_equivalent_tflops": f / (ms_d * 1e-3) / 1e12,
          "rel_diff_vs_fp64": float((y - y64).abs().max() / y64.abs().max())}
    return {"workload": f"DG Stokes, {n_cells}^3 affine cells, velocity Q{k} x3 + pressure Q{k - 1}, FP64",
            "ndofs": op.ndofs, "dof_s": op.ndofs / (ms * 1e-3), "ms": ms, "kernel_ms": kt,
            "tflops_model": f / (ms * 1e-3) / 1e12, "frac_fp64_peak_model": f / (ms * 1e-3) / 1e12 / pk["fp64_tflops"],
            "df64": df}


def adjoint_apply(n_cells=64, k=3):
    """Config 5: adjoint (A^T r and dL/dkappa at every point) on 64^3 trilinear cells, Q3,
    log-normal kappa; geometry recomputed in the kernels."""
    import torch
    from paper_1812_08075_gb300 import dg
    n = (n_cells,) * 3
    op = dg.Operator(dg.Mesh(*n, wl.perturbed_vertices(*n, seed=1)), k)
    kv, kf = wl.lognormal_kappa(op.mesh.ncell, k + 1, seed=2)
    tkv, tkf = torch.from_numpy(kv).cuda(), torch.from_numpy(kf).cuda()
    op.set_kappa(tkv, tkf)
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 3)).cuda()
    r = torch.from_numpy(wl.uniform_vector(op.ndofs, 4)).cuda()
    y = torch.empty_like(x)
    gv, gf = torch.empty_like(tkv), torch.empty_like(tkf)
    ms_fwd, _, _ = time_applies(op, x, y, 20, 3, None, profile=False)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        dg.dg_apply_adjoint(op.handle, r.data_ptr(), x.data_ptr(), y.data_ptr(), gv.data_ptr(), gf.data_ptr(),
                            stream.cuda_stream, nrhs=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        dg.dg_apply_adjoint(op.handle, r.data_ptr(), x.data_ptr(), y.data_ptr(), gv.data_ptr(), gf.data_ptr(),
                            stream.cuda_stream, nrhs=1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1) / 20
    # the same adjoint in double-float arithmetic (DG_VARIANT_DF64)
    ref = (y.clone(), gv.clone(), gf.clone())
    op.set_variant(dg.DG_VARIANT_DF64)
    adj = lambda: dg.dg_apply_adjoint(op.handle, r.data_ptr(), x.data_ptr(), y.data_ptr(), gv.data_ptr(),  # noqa: E731
                                      gf.data_ptr(), stream.cuda_stream, nrhs=1)
    ms_adj_df = event_ms(adj)
    diffs = [float((q - p).abs().max() / p.abs().max()) for p, q in zip(ref, (y, gv, gf))]
    ms_fwd_df, _, _ = time_applies(op, x, y, 20, 3, None, profile=False)
    return {"workload": f"{n_cells}^3 trilinear cells, Q{k}, log-normal kappa at every point, FP64",
            "ndofs": op.ndofs, "forward_ms": ms_fwd, "adjoint_ms": ms_adj,
            "adjoint_dof_s": op.ndofs / (ms_adj * 1e-3), "geometry": "recomputed in the adjoint kernels",
            "df64": {"forward_ms": ms_fwd_df, "adjoint_ms": ms_adj_df, "speedup_adjoint": ms_adj / ms_adj_df,
                     "rel_diff_vs_fp64": {"y": diffs[0], "dkappa_vol": diffs[1], "dkappa_face": diffs[2]}}}


def event_ms(fn, reps=20, warm=3):
    """Mean CUDA-event milliseconds of fn() on the current stream."""
    import torch
    for _ in range(warm):
        fn()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def next_rows_apply(n_cells=64, k=3):
    """The widened rows on config 5's mesh (64^3 trilinear, Q3, FP64): the residual's data
    terms (dg_rhs), the semilinear reaction's residual operator and Jacobian action
    (dg_apply_semilinear), and the cell-block Jacobi preconditioner on the affine mesh."""
    import torch
    from paper_1812_08075_gb300 import dg
    n = (n_cells,) * 3
    op = dg.Operator(dg.Mesh(*n, wl.perturbed_vertices(*n, seed=1)), k)
    m = k + 1
    u0 = torch.from_numpy(wl.uniform_vector(op.ndofs, 3)).cuda()
    w = torch.from_numpy(wl.uniform_vector(op.ndofs, 4)).cuda()
    f = torch.from_numpy(wl.uniform_vector(op.mesh.ncell * m ** 3, 5)).cuda()
    g = torch.from_numpy(wl.uniform_vector(op.mesh.ncell * 6 * m ** 2, 6)).cuda()
    y = torch.empty_like(w)
    ms_fwd = event_ms(lambda: op.apply(w, y))
    ms_rhs = event_ms(lambda: op.rhs(f, g))
    ms_res = event_ms(lambda: op.semilinear(w, 2.0))
    ms_jac = event_ms(lambda: op.semilinear(w, 2.0, u0=u0))
    aff = dg.Operator(dg.Mesh(*n), k)
    ms_bj = event_ms(lambda: aff.block_jacobi(w, y))
    aff32 = dg.Operator(dg.Mesh(*n), k, precision=dg.DG_FP32)
    w32, y32 = w.float(), torch.empty_like(w.float())
    ms_bj32 = event_ms(lambda: aff32.block_jacobi(w32, y32))
    # anisotropic degrees and quadrature on the trilinear mesh (geometry recomputed)
    aniso = {}
    for prec, tag in ((dg.DG_FP64, "fp64"), (dg.DG_FP32, "fp32")):
        an = dg.Operator(op.mesh, 0, degrees=(1, 3, 2), quad=(3, 4, 3), precision=prec)
        xa = torch.from_numpy(wl.uniform_vector(an.ndofs, 7)).to("cuda", an.dtype)
        ya = torch.empty_like(xa)
        ms_a = event_ms(lambda: an.apply(xa, ya))
        aniso[tag] = {"ms": ms_a, "dof_s": an.ndofs / (ms_a * 1e-3)}
        del an, xa, ya
    return {"workload": f"{n_cells}^3 trilinear cells (block Jacobi: affine), Q{k}, FP64 unless stated",
            "ndofs": op.ndofs, "forward_apply_ms": ms_fwd, "rhs_ms": ms_rhs,
            "semilinear_residual_ms": ms_res, "semilinear_jacobian_ms": ms_jac,
            "block_jacobi_fp64_ms": ms_bj, "block_jacobi_fp32_ms": ms_bj32,
            "aniso_k132_m343_trilinear": aniso,
            "note": "semilinear and rhs recompute the geometry in the kernels; the forward apply reads stored geometry"}


def solve_entry(n, k, nrhs, rtol, inner_rtol=1e-3, delta=0.1, fp64_max_iters=20000, precond=2,
                fp64_preconds=(0, 2)):
    """Config 4's solve to rtol, all right-hand sides advanced together: mixed CG with
    reliable updates (FP32 iterations, FP64 residual replacements), FP64 iterative
    refinement around FP32 CG, and the all-FP64 CG with each preconditioner of
    fp64_preconds, on the same right-hand sides. Wall seconds of each solve call
    (synchronous), its iterations, and the FP64 residual recomputed afterwards."""
    import torch
    from paper_1812_08075_gb300 import dg
    mesh = dg.Mesh(n, n, n)
    op64 = dg.Operator(mesh, k, max_rhs=nrhs)
    op32 = dg.Operator(mesh, k, precision=dg.DG_FP32, max_rhs=nrhs)
    b = config4_rhs(op64, n, k, nrhs)
    stream = torch.cuda.current_stream().cuda_stream
    # both operators take the variant and blocking the framework's tuner measures fastest
    # for nrhs right-hand sides, so the all-FP64 CG runs on its best apply too
    tune64, tune32 = op64.autotune(nrhs), op32.autotune(nrhs)
    out = {"workload": f"scalar SIPG, {n}^3 affine cells, Q{k}, {nrhs} right-hand sides (Gauss-projected "
                       f"sin-product load vector + U[-1,1] noise), x0 = 0",
           "ndofs": op64.ndofs, "nrhs": nrhs, "rtol": rtol,
           "fp64_operator": {"variant": VARIANT_NAMES[op64.stats().variant], "apply_ms": tune64["ms_best"]},
           "fp32_operator": {"variant": VARIANT_NAMES[op32.stats().variant], "apply_ms": tune32["ms_best"]},
           "mixed_preconditioner": PRECOND_NAMES[precond]}
    # set up the preconditioners and the FP32 operator's variant before timing
    for op, pcs, bb in ((op64, fp64_preconds, b), (op32, (precond,), b.float())):
        for pc in pcs:
            if pc:
                xz = torch.zeros_like(bb)
                dg.dg_cg_solve(op.handle, bb.data_ptr(), xz.data_ptr(), nrhs, dg.dg_cg_options(1e-1, 50, 50, 0, pc),
                               stream)
                del xz

    def relres(x):
        r = b - op64.apply(x)
        return max(float(torch.linalg.norm(r[i]) / torch.linalg.norm(b[i])) for i in range(nrhs))

    def timed(fn):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ok, info = fn(x)
        torch.cuda.synchronize()
        return time.perf_counter() - t, ok, info, relres(x)

    sec, ok, info, rr = timed(lambda x: dg.dg_mixed_cg_solve(
        op64.handle, op32.handle, b.data_ptr(), x.data_ptr(), nrhs, delta,
        dg.dg_cg_options(rtol, 100000, 50, 1, precond), stream))
    out["mixed_reliable"] = {"seconds": sec, "converged": ok, "fp32_iters_max": max(i["iters"] for i in info),
                             "fp64_updates_max": max(i["outer"] for i in info), "relres_fp64_max": rr, "delta": delta}
    sec, ok, info, rr = timed(lambda x: dg.dg_refine_solve(
        op64.handle, op32.handle, b.data_ptr(), x.data_ptr(), nrhs, rtol, 30,
        dg.dg_cg_options(inner_rtol, 100000, 50, 1, precond), stream))
    out["refinement"] = {"seconds": sec, "converged": ok, "outer_max": max(i["outer"] for i in info),
                         "inner_iters_max": max(i["iters"] for i in info), "relres_fp64_max": rr,
                         "inner_rtol": inner_rtol}
    best = None
    for pc in fp64_preconds:
        sec, ok, info, rr = timed(lambda x: dg.dg_cg_solve(
            op64.handle, b.data_ptr(), x.data_ptr(), nrhs, dg.dg_cg_options(rtol, fp64_max_iters, 50, 1, pc), stream))
        out[f"fp64_cg_{['none', 'jacobi', 'block_jacobi'][pc]}"] = {
            "seconds": sec, "converged": ok, "iters_max": max(i["iters"] for i in info), "relres_fp64_max": rr,
            "preconditioner": PRECOND_NAMES[pc]}
        if ok and (best is None or sec < best[0]):
            best = (sec, pc)
    if best:
        out["fp64_cg_best_seconds"] = best[0]
        out["fp64_cg_best_preconditioner"] = PRECOND_NAMES[best[1]]
        out["speedup_mixed_reliable_over_best_fp64"] = best[0] / out["mixed_reliable"]["seconds"]
        out["speedup_refinement_over_best_fp64"] = best[0] / out["refinement"]["seconds"]
    return out


def run_solve(args):
    """Config 4's solve comparison alone (sizes from the command line)."""
    from paper_1812_08075_gb300 import build as libbuild
    libbuild.build()
    pcs = (args.precond_fp64,) if args.precond_fp64 is not None else (0, 2)
    out = solve_entry(args.solve_cells, args.solve_degree, args.solve_rhs, args.solve_rtol, args.inner_rtol,
                      args.delta, args.fp64_max_iters, args.precond, pcs)
    out["mode"] = "solve"
    print(json.dumps(out), flush=True)


def df64_entry(op, x, y64, pk, args):
    """The benchmark operator in double-float arithmetic (DG_VARIANT_DF64): its three
    kernels on the FP32 pipes with FP64 vectors; y64 holds the FP64 variant's A x."""
    import torch
    from paper_1812_08075_gb300 import dg
    op.set_variant(dg.DG_VARIANT_DF64)
    tuning = op.autotune(1) if args.autotune else None
    y = torch.empty_like(y64)
    ms, kt, _ = time_applies(op, x, y, min(args.steps, 100), 5, None, profile=True)
    f = sum(op.stats().flops)
    return {"variant": "double-float three-kernel (pairs of FP32, 48-bit significand)",
            "dof_s": op.ndofs / (ms * 1e-3), "ms_per_apply": ms, "kernel_ms": kt,
            "fp64_equivalent_tflops": f / (ms * 1e-3) / 1e12,
            "fp64_equivalent_frac_of_fp64_peak": f / (ms * 1e-3) / 1e12 / pk["fp64_tflops"],
            "rel_diff_vs_fp64": float((y - y64).abs().max() / y64.abs().max()),
            "tuning": tuning}


def run_ours(args, rank, world, dist):
    import torch
    from paper_1812_08075_gb300 import build as libbuild, dg
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if local == 0:
        libbuild.build()
    if dist:
        dist.barrier()
    k = args.degree
    n = (N_CELLS,) * 3
    verts = wl.perturbed_vertices(*n, seed=1)
    mesh = dg.Mesh(*n, verts)
    op = dg.Operator(mesh, k)
    tuning = op.autotune(1) if args.autotune else None
    x = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).cuda()
    y = torch.empty_like(x)
    pk = peaks(probe=rank == 0)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    ms, kt, (t0, t1) = time_applies(op, x, y, args.steps, args.warmup, dist, profile=True)
    clocks = sampler.stop(t0, t1) if sampler else None
    ms_all, value = aggregate(ms, op.ndofs, world, dist)
    st = op.stats()
    flops = list(st.flops)
    names = ["k_cell (volume: interpolate, gradient, pointwise, transposed derivative; face traces)",
             "k_face (interior and boundary face terms)", "k_back (face lifting and transposed interpolation)"]
    dom = int(np.argmax(kt))
    achieved = flops[dom] / (kt[dom] * 1e-3) / 1e12
    traffic = (KCELL_Q3_DRAM_BYTES_PER_CELL * op.mesh.ncell) if (k == 3 and dom == 0) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
                "frac": achieved / pk["fp64_tflops"], "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_cell at 40^3 Q3, "
                                  "scaled by cells to this launch" if traffic else None,
                "algorithmic_bytes_per_launch": st.bytes[dom],
                "kernel": names[dom], "kernel_ms": kt[dom],
                "peak_source": f"FP64 CUDA-core peak derived: {pk['sms']} SMs x 2 DFMA/clk x 2 flop x "
                               f"{pk['clk_mhz']:.0f} MHz (1.25 TFLOP/s nominal); this run's FMA-chain probe "
                               f"(dg_measure_fma_peak) measured {pk.get('fp64_probe_tflops', float('nan')):.3f}",
                "probe_tflops": pk.get("fp64_probe_tflops"),
                "frac_of_probe": achieved / pk["fp64_probe_tflops"] if pk.get("fp64_probe_tflops") else None,
                "algorithmic_flops_per_launch": flops[dom]}
    tot_flops = sum(flops)
    whole = {"flops_per_apply": tot_flops, "tflops": tot_flops / (ms * 1e-3) / 1e12,
             "frac_fp64_peak": tot_flops / (ms * 1e-3) / 1e12 / pk["fp64_tflops"],
             "kernel_ms": {"k_cell": kt[0], "k_face": kt[1], "k_back": kt[2]},
             "hbm_bytes_algorithmic": st.dofs_bytes, "gb_s_algorithmic": st.dofs_bytes / (ms * 1e-3) / 1e9}
    out = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(k),
           "roofline": roofline, "apply": whole,
           "gpu_launches": (3 if st.variant == dg.DG_VARIANT_THREE_KERNEL else 1) * args.steps, "clocks": clocks,
           "tuning": tuning}
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    xh = torch.from_numpy(wl.uniform_vector(op.ndofs, 0)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        op.apply_host(xh, yh)
    e2e_steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        op.apply_host(xh, yh)
    dt = (time.perf_counter() - t) / e2e_steps
    out["e2e"] = {"value": world * op.ndofs / dt, "unit": "DOF/s", "h2d_bytes_per_step": 8 * op.ndofs,
                  "d2h_bytes_per_step": 8 * op.ndofs, "steps": e2e_steps, "api": "dg_apply_host (pinned host x, y)"}
    if rank == 0:
        out["df64"] = df64_entry(op, x, y, pk, args)
    del op, x, y, xh, yh
    if args.sweep and rank == 0:
        sweep = {}
        vert_bytes = 8 * 3 * (N_CELLS + 1) ** 3  # vertex coordinates, read by the geometry
        for kk in (1, 2, 3, 4, 5):
            y64 = None
            for prec, tag, es in ((dg.DG_FP64, "fp64", 8), (dg.DG_FP32, "fp32", 4)):
                o = dg.Operator(mesh, kk, precision=prec)
                if args.autotune:  # the framework's own tuner, as for the headline operator
                    o.autotune(1)
                xx = torch.from_numpy(wl.uniform_vector(o.ndofs, 0)).to("cuda", o.dtype)
                yy = torch.empty_like(xx)
                ms_k, kt_k, _ = time_applies(o, xx, yy, 10, 3, None, profile=True)
                st_k = o.stats()
                ent = {"dof_s": o.ndofs / (ms_k * 1e-3), "ms": ms_k, "kernel_ms": kt_k,
                       "blocking": [st_k.variant, st_k.cells_per_block, st_k.faces_per_block],
                       "geometry": "recomputed in the kernels" if st_k.geometry == dg.DG_GEOM_RECOMPUTE
                       else "stored per point"}
                ent.update(roofline_entry(sum(st_k.flops), 2 * es * o.ndofs + vert_bytes, ms_k, pk,
                                          prec == dg.DG_FP32, impl_bytes=sum(st_k.bytes)))
                if prec == dg.DG_FP32:  # error of the FP32 result against the FP64 apply of the same x
                    ent["err_vs_fp64"] = float((yy.double() - y64).abs().max() / y64.abs().max())
                sweep[f"Q{kk}_{tag}"] = ent
                if prec == dg.DG_FP64:  # the same operator in double-float arithmetic, blockings tuned
                    y64 = yy.clone()
                    f = sum(st_k.flops)
                    o.set_variant(dg.DG_VARIANT_DF64)
                    if args.autotune:
                        o.autotune(1)
                    ms_d, kt_d, _ = time_applies(o, xx, yy, 10, 3, None, profile=True)
                    ent_d = {"dof_s": o.ndofs / (ms_d * 1e-3), "ms": ms_d,
                             "fp64_equivalent_tflops": f / (ms_d * 1e-3) / 1e12,
                             "speedup_over_fp64": ms_k / ms_d,
                             "err_vs_fp64": float((yy - y64).abs().max() / y64.abs().max()),
                             "kernel_ms": kt_d}
                    # double-float runs on the FP32 pipes with about ten FP32 operations per FP64
                    # one, so its rate is quoted as FP64-equivalent work, beside its HBM fraction
                    ent_d["alg_bytes"] = 16 * o.ndofs + vert_bytes
                    ent_d["frac_hbm_alg"] = ent_d["alg_bytes"] / (ms_d * 1e-3) / 1e9 / pk["hbm_gbs"]
                    sweep[f"Q{kk}_df64"] = ent_d
                del o, xx, yy
            del y64
        out["sweep"] = sweep
    if args.mixed and rank == 0:
        out["mixed_apply"] = mixed_apply(pk, n_cells=args.mixed_cells)
    if args.sweep and rank == 0:
        out["stokes"] = stokes_apply(pk)
        out["adjoint"] = adjoint_apply()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = host_cores()
        rate, ncells, dt = oracle_rate(k, 15.0, cores)
        out["cpu_baseline"] = {"value": rate, "unit": "DOF/s", "cores": cores, "kind": "oracle",
                               "sample": f"{ncells} random cells of the {N_CELLS}^3 Q{k} workload, cell-gather "
                                         f"form, {dt:.1f} s wall on {cores} threads"}
    if args.solve and rank == 0 and world == 1:
        torch.cuda.empty_cache()
        out["solve"] = solve_entry(args.solve_cells, args.solve_degree, args.solve_rhs, args.solve_rtol,
                                   args.inner_rtol, args.delta, args.fp64_max_iters, args.precond,
                                   (0, 2) if args.precond_fp64 is None else (args.precond_fp64,))
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--sweep", dest="sweep", action="store_true", default=True)
    ap.add_argument("--no-sweep", dest="sweep", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=64, help="cells per axis (64 is the benchmark workload)")
    ap.add_argument("--mode", default="apply", choices=["apply", "solve", "extras"])
    ap.add_argument("--stokes-cells", type=int, default=32)
    ap.add_argument("--adjoint-cells", type=int, default=64)
    ap.add_argument("--no-mixed", dest="mixed", action="store_false", default=True)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", default=True)
    ap.add_argument("--mixed-cells", type=int, default=128, help="cells per axis of the mixed-precision apply")
    ap.add_argument("--solve-cells", type=int, default=128)
    ap.add_argument("--solve-degree", type=int, default=2)
    ap.add_argument("--solve-rhs", type=int, default=16)
    ap.add_argument("--solve-rtol", type=float, default=1e-10)
    ap.add_argument("--inner-rtol", type=float, default=1e-3)
    ap.add_argument("--fp64-max-iters", type=int, default=20000)
    ap.add_argument("--precond", type=int, default=2, choices=(0, 1, 2),
                    help="preconditioner of the mixed solvers: 0 none, 1 point Jacobi, 2 cell-block Jacobi")
    ap.add_argument("--delta", type=float, default=0.1,
                    help="reliable-update threshold of the mixed CG (FP32 residual reduction per update)")
    ap.add_argument("--precond-fp64", type=int, default=None, choices=(0, 1, 2),
                    help="one preconditioner for the FP64 CG (default: time it with none and with block Jacobi)")
    ap.add_argument("--no-solve", dest="solve", action="store_false", default=True,
                    help="skip config 4's solve comparison (mixed vs FP64 CG) of the default run")
    args = ap.parse_args()
    global N_CELLS
    N_CELLS = args.cells
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = tdist
    if args.mode == "solve":
        if rank == 0:
            run_solve(args)
    elif args.mode == "extras":
        if rank == 0:
            import torch
            from paper_1812_08075_gb300 import build as libbuild
            libbuild.build()
            print(json.dumps({"mode": "extras", "stokes": stokes_apply(peaks(), n_cells=args.stokes_cells),
                              "adjoint": adjoint_apply(n_cells=args.adjoint_cells),
                              "next_rows": next_rows_apply(n_cells=args.adjoint_cells)}), flush=True)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
