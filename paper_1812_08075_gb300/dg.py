"""Thin ctypes binding of libdg's C ABI (include/dg.h).

Functions named like the C entry points marshal arguments and raise ``DGError`` on a
non-zero status; every step of an apply runs in the library's CUDA kernels. ``Mesh``
and ``Operator`` wrap the handles for PyTorch callers (device memory and streams come
from torch). Importing this module does not build or load anything; the first call
loads ``_build/libdg_sm103a.so`` and raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdg_sm103a.so")

DG_OK, DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NOT_CONVERGED, DG_ERR_TIMEOUT = range(7)
DG_PEN_CONFIG, DG_PEN_PAPER = 0, 1
DG_SCALAR, DG_STOKES = 0, 1
DG_FP64, DG_FP32 = 0, 1
DG_GEOM_AUTO, DG_GEOM_STORED, DG_GEOM_RECOMPUTE = 0, 1, 2
DG_VARIANT_AUTO, DG_VARIANT_THREE_KERNEL, DG_VARIANT_FUSED, DG_VARIANT_CELLWISE, DG_VARIANT_DF64 = 0, 1, 2, 3, 4
DG_PRECOND_NONE, DG_PRECOND_JACOBI, DG_PRECOND_BLOCK_JACOBI = 0, 1, 2
DG_SEMILINEAR_RESIDUAL, DG_SEMILINEAR_JACOBIAN = 1, 2

EXPORTED = [
    "dg_status_string", "dg_get_last_error", "dg_mesh_create", "dg_mesh_destroy", "dg_operator_create",
    "dg_operator_destroy", "dg_operator_ndofs", "dg_operator_stats", "dg_operator_set_kappa", "dg_apply",
    "dg_apply_host", "dg_apply_adjoint", "dg_reference_tables", "dg_operator_profile", "dg_operator_kernel_times",
    "dg_apply_affine_static", "dg_cg_solve", "dg_refine_solve", "dg_operator_set_variant",
    "dg_operator_autotune", "dg_rhs", "dg_operator_diagonal", "dg_operator_block_jacobi",
    "dg_operator_predict", "dg_operator_time", "dg_operator_autotune_prior", "dg_apply_semilinear",
    "dg_operator_create_aniso", "dg_mixed_cg_solve", "dg_measure_fma_peak",
    "dg_measure_mma_peak", "dg_device_faults",
]


class DGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


class dg_penalty(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("reserved", ctypes.c_int32), ("alpha", ctypes.c_double)]


class dg_coefficients(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_int32), ("precision", ctypes.c_int32), ("dirichlet_mask", ctypes.c_int32),
                ("max_rhs", ctypes.c_int32), ("geometry", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("c", ctypes.c_double), ("mu", ctypes.c_double), ("theta", ctypes.c_double)]


class dg_cg_options(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("precond", ctypes.c_int32)]


class dg_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("breakdown", ctypes.c_int32), ("relres", ctypes.c_double)]


class dg_tune_result(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("cells_per_block", ctypes.c_int32), ("faces_per_block", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("ms_best", ctypes.c_double), ("ms_default", ctypes.c_double)]


class dg_stats(ctypes.Structure):
    _fields_ = [("ndofs", ctypes.c_int64), ("ncell", ctypes.c_int64), ("nface", ctypes.c_int64),
                ("flops", ctypes.c_double * 3), ("bytes", ctypes.c_double * 3), ("dofs_bytes", ctypes.c_double),
                ("cells_per_block", ctypes.c_int32), ("faces_per_block", ctypes.c_int32),
                ("threads_cell", ctypes.c_int32), ("threads_face", ctypes.c_int32),
                ("geometry", ctypes.c_int32), ("variant", ctypes.c_int32), ("persistent_grid", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded libdg (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdg is not built ({LIB_PATH} missing); run paper_1812_08075_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        L.dg_status_string.restype = ctypes.c_char_p
        L.dg_status_string.argtypes = [i32]
        L.dg_get_last_error.restype = i32
        L.dg_mesh_create.argtypes = [i32, i32, i32, vp, ctypes.POINTER(vp)]
        L.dg_mesh_destroy.argtypes = [vp]
        L.dg_operator_create.argtypes = [vp, i32, i32, ctypes.POINTER(dg_penalty), ctypes.POINTER(dg_coefficients),
                                         ctypes.POINTER(vp)]
        L.dg_operator_destroy.argtypes = [vp]
        L.dg_operator_ndofs.argtypes = [vp, ctypes.POINTER(i64)]
        L.dg_operator_stats.argtypes = [vp, ctypes.POINTER(dg_stats)]
        L.dg_operator_set_kappa.argtypes = [vp, vp, vp]
        L.dg_apply.argtypes = [vp, vp, vp, i32, vp]
        L.dg_apply_host.argtypes = [vp, vp, vp, i32, vp]
        L.dg_apply_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
        L.dg_reference_tables.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.dg_operator_profile.argtypes = [vp, i32]
        L.dg_operator_set_variant.argtypes = [vp, i32, i32, i32]
        L.dg_rhs.argtypes = [vp, vp, vp, vp, vp]
        L.dg_operator_diagonal.argtypes = [vp, vp, vp]
        L.dg_operator_block_jacobi.argtypes = [vp, vp, vp, i32, vp]
        L.dg_operator_create_aniso.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(dg_penalty), ctypes.POINTER(dg_coefficients),
                                               ctypes.POINTER(ctypes.c_void_p)]
        L.dg_apply_semilinear.argtypes = [vp, i32, ctypes.c_double, vp, vp, vp, vp]
        L.dg_operator_predict.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_double)]
        L.dg_operator_time.argtypes = [vp, i32, i32, i32, i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.dg_operator_autotune_prior.argtypes = [vp, i32, i32, vp, ctypes.POINTER(dg_tune_result)]
        L.dg_operator_autotune.argtypes = [vp, i32, vp, ctypes.POINTER(dg_tune_result)]
        L.dg_cg_solve.argtypes = [vp, vp, vp, i32, ctypes.POINTER(dg_cg_options), ctypes.POINTER(dg_solve_info), vp]
        L.dg_mixed_cg_solve.argtypes = [vp, vp, vp, vp, i32, ctypes.c_double, ctypes.POINTER(dg_cg_options),
                                        ctypes.POINTER(dg_solve_info), vp]
        L.dg_refine_solve.argtypes = [vp, vp, vp, vp, i32, ctypes.c_double, i32, ctypes.POINTER(dg_cg_options),
                                      ctypes.POINTER(dg_solve_info), vp]
        L.dg_apply_affine_static.argtypes = [i32, i32, i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             i32, vp, vp, vp]
        L.dg_measure_fma_peak.argtypes = [i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.dg_measure_mma_peak.argtypes = [i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.dg_device_faults.argtypes = [i32, ctypes.POINTER(ctypes.c_uint)]
        L.dg_operator_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double * 3), ctypes.POINTER(i64)]
        for name in EXPORTED:
            if name not in ("dg_status_string",):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != DG_OK:
        raise DGError(status, where)


def status_string(status: int) -> str:
    return lib().dg_status_string(status).decode()


# ------------------------------------------------------------ C-ABI named wrappers

def dg_mesh_create(nx: int, ny: int, nz: int, vertices: Optional[np.ndarray] = None) -> int:
    h = ctypes.c_void_p()
    v = None
    if vertices is not None:
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        if v.shape != ((nx + 1) * (ny + 1) * (nz + 1), 3):
            raise ValueError("vertices must have shape [(nx+1)(ny+1)(nz+1), 3]")
    _check(lib().dg_mesh_create(nx, ny, nz, None if v is None else v.ctypes.data, ctypes.byref(h)), "dg_mesh_create")
    return h.value


def dg_mesh_destroy(mesh: int):
    lib().dg_mesh_destroy(mesh)


def dg_operator_create(mesh: int, degree: int, quad_points_1d: int, penalty: dg_penalty,
                       coef: dg_coefficients) -> int:
    h = ctypes.c_void_p()
    _check(lib().dg_operator_create(mesh, degree, quad_points_1d, ctypes.byref(penalty), ctypes.byref(coef),
                                    ctypes.byref(h)), "dg_operator_create")
    return h.value


def dg_operator_create_aniso(mesh: int, degrees, penalty: dg_penalty, coef: dg_coefficients, quad=None) -> int:
    h = ctypes.c_void_p()
    ks = (ctypes.c_int32 * 3)(*degrees)
    qs = None if quad is None else (ctypes.c_int32 * 3)(*quad)
    _check(lib().dg_operator_create_aniso(mesh, ks, qs, ctypes.byref(penalty), ctypes.byref(coef), ctypes.byref(h)),
           "dg_operator_create_aniso")
    return h.value


def dg_operator_destroy(op: int):
    lib().dg_operator_destroy(op)


def dg_operator_ndofs(op: int) -> int:
    n = ctypes.c_int64()
    _check(lib().dg_operator_ndofs(op, ctypes.byref(n)), "dg_operator_ndofs")
    return n.value


def dg_operator_stats(op: int) -> dg_stats:
    s = dg_stats()
    _check(lib().dg_operator_stats(op, ctypes.byref(s)), "dg_operator_stats")
    return s


def dg_operator_set_kappa(op: int, kappa_vol_ptr: Optional[int], kappa_face_ptr: Optional[int]):
    _check(lib().dg_operator_set_kappa(op, kappa_vol_ptr, kappa_face_ptr), "dg_operator_set_kappa")


def dg_apply(op: int, x_ptr: int, y_ptr: int, nrhs: int, stream: Optional[int]):
    _check(lib().dg_apply(op, x_ptr, y_ptr, nrhs, stream), "dg_apply")


def dg_apply_host(op: int, x_ptr: int, y_ptr: int, nrhs: int, stream: Optional[int]):
    _check(lib().dg_apply_host(op, x_ptr, y_ptr, nrhs, stream), "dg_apply_host")


def dg_apply_adjoint(op: int, r_ptr: int, x_ptr: Optional[int], y_ptr: int, dk_vol_ptr: Optional[int],
                     dk_face_ptr: Optional[int], stream: Optional[int], nrhs: int = 1):
    """y_s = A^T r_s for nrhs vectors; dkappa summed over the right-hand sides."""
    _check(lib().dg_apply_adjoint(op, r_ptr, x_ptr, y_ptr, dk_vol_ptr, dk_face_ptr, nrhs, stream),
           "dg_apply_adjoint")


def dg_apply_affine_static(nx: int, ny: int, nz: int, degree: int, c: float, theta: float, penalty_alpha: float,
                           dirichlet_mask: int, x_ptr: int, y_ptr: int, stream: Optional[int]):
    """FP64 affine apply that allocates nothing (its scratch is a fixed 32 MiB device array)."""
    _check(lib().dg_apply_affine_static(nx, ny, nz, degree, c, theta, penalty_alpha, dirichlet_mask, x_ptr, y_ptr,
                                        stream), "dg_apply_affine_static")


def _solve_result(status, infos, where):
    out = [dict(iters=i.iters, outer=i.outer, converged=bool(i.converged), breakdown=bool(i.breakdown),
                relres=i.relres) for i in infos]
    if status not in (DG_OK, DG_ERR_NOT_CONVERGED):
        raise DGError(status, where)
    return status == DG_OK, out


def dg_cg_solve(op: int, b_ptr: int, x_ptr: int, nrhs: int, opt: dg_cg_options, stream: Optional[int]):
    """Returns (all converged, per right-hand-side info dicts)."""
    infos = (dg_solve_info * nrhs)()
    st = lib().dg_cg_solve(op, b_ptr, x_ptr, nrhs, ctypes.byref(opt), infos, stream)
    return _solve_result(st, infos, "dg_cg_solve")


def dg_mixed_cg_solve(op64: int, op32: int, b_ptr: int, x_ptr: int, nrhs: int, delta: float, opt: dg_cg_options,
                      stream: Optional[int]):
    """Mixed-precision CG with reliable updates: (ok, infos); raises on errors other than
    non-convergence."""
    infos = (dg_solve_info * nrhs)()
    st = lib().dg_mixed_cg_solve(op64, op32, b_ptr, x_ptr, nrhs, delta, ctypes.byref(opt), infos, stream)
    return _solve_result(st, infos, "dg_mixed_cg_solve")


def dg_refine_solve(op64: int, op32: int, b_ptr: int, x_ptr: int, nrhs: int, rtol: float, max_outer: int,
                    inner: dg_cg_options, stream: Optional[int]):
    """Returns (all converged, per right-hand-side info dicts)."""
    infos = (dg_solve_info * nrhs)()
    st = lib().dg_refine_solve(op64, op32, b_ptr, x_ptr, nrhs, rtol, max_outer, ctypes.byref(inner), infos, stream)
    return _solve_result(st, infos, "dg_refine_solve")


def dg_operator_set_variant(op: int, variant: int, cells_per_block: int = 0, faces_per_block: int = 0):
    _check(lib().dg_operator_set_variant(op, variant, cells_per_block, faces_per_block), "dg_operator_set_variant")


def dg_operator_autotune(op: int, nrhs: int, stream: Optional[int]) -> dict:
    r = dg_tune_result()
    _check(lib().dg_operator_autotune(op, nrhs, stream, ctypes.byref(r)), "dg_operator_autotune")
    return {f: getattr(r, f) for f, _ in dg_tune_result._fields_}


def dg_rhs(op: int, f_ptr: Optional[int], g_ptr: Optional[int], F_ptr: int, stream: Optional[int]):
    _check(lib().dg_rhs(op, f_ptr, g_ptr, F_ptr, stream), "dg_rhs")


def dg_operator_diagonal(op: int, diag_ptr: int, stream: Optional[int]):
    _check(lib().dg_operator_diagonal(op, diag_ptr, stream), "dg_operator_diagonal")


def dg_operator_block_jacobi(op: int, r_ptr: int, z_ptr: int, nrhs: int, stream: Optional[int]):
    _check(lib().dg_operator_block_jacobi(op, r_ptr, z_ptr, nrhs, stream), "dg_operator_block_jacobi")


def dg_operator_predict(op: int, nrhs: int, variant: int, cells_per_block: int, faces_per_block: int = 0) -> float:
    ms = ctypes.c_double()
    _check(lib().dg_operator_predict(op, nrhs, variant, cells_per_block, faces_per_block, ctypes.byref(ms)),
           "dg_operator_predict")
    return ms.value


def dg_operator_time(op: int, nrhs: int, variant: int, cells_per_block: int, faces_per_block: int = 0,
                     stream: Optional[int] = None) -> float:
    ms = ctypes.c_double()
    _check(lib().dg_operator_time(op, nrhs, variant, cells_per_block, faces_per_block, stream, ctypes.byref(ms)),
           "dg_operator_time")
    return ms.value


def dg_operator_autotune_prior(op: int, nrhs: int, measure: int, stream: Optional[int] = None):
    r = dg_tune_result()
    _check(lib().dg_operator_autotune_prior(op, nrhs, measure, stream, ctypes.byref(r)), "dg_operator_autotune_prior")
    return {f: getattr(r, f) for f, _ in dg_tune_result._fields_}


def dg_operator_profile(op: int, enable: bool):
    _check(lib().dg_operator_profile(op, int(enable)), "dg_operator_profile")


def dg_operator_kernel_times(op: int):
    """(milliseconds per kernel summed over the recorded applies, number of applies)."""
    ms = (ctypes.c_double * 3)()
    n = ctypes.c_int64()
    _check(lib().dg_operator_kernel_times(op, ctypes.byref(ms), ctypes.byref(n)), "dg_operator_kernel_times")
    return list(ms), n.value


def dg_measure_fma_peak(precision: int, stream: Optional[int] = None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current GPU in FP64 or FP32."""
    t = ctypes.c_double()
    _check(lib().dg_measure_fma_peak(precision, stream, ctypes.byref(t)), "dg_measure_fma_peak")
    return t.value


def dg_measure_mma_peak(kind: int, stream: Optional[int] = None) -> float:
    """Measured tensor-core throughput (TFLOP/s): kind 0 FP64 DMMA m8n8k4, 1 TF32 m16n8k8,
    2 DMMA and DFMA issued together."""
    t = ctypes.c_double()
    _check(lib().dg_measure_mma_peak(kind, stream, ctypes.byref(t)), "dg_measure_mma_peak")
    return t.value


def dg_device_faults(clear: bool = True) -> int:
    """Bit mask of device-side faults recorded since the last clear (0 if none): bit 0, a
    cellwise kernel's wait for its bulk copies gave up."""
    v = ctypes.c_uint()
    _check(lib().dg_device_faults(int(clear), ctypes.byref(v)), "dg_device_faults")
    return v.value


def dg_reference_tables(degree: int, m: int = 0):
    m = m or degree + 1
    out = {k: np.zeros(n) for k, n in (("gauss_nodes", m), ("gauss_weights", m), ("gll_nodes", degree + 1),
                                       ("interp", m * (degree + 1)), ("dcol", m * m), ("end_val", 2 * m),
                                       ("end_der", 2 * m))}
    _check(lib().dg_reference_tables(degree, m, *(out[k].ctypes.data for k in
                                                  ("gauss_nodes", "gauss_weights", "gll_nodes", "interp", "dcol",
                                                   "end_val", "end_der"))), "dg_reference_tables")
    out["interp"] = out["interp"].reshape(m, degree + 1)
    out["dcol"] = out["dcol"].reshape(m, m)
    out["end_val"] = out["end_val"].reshape(2, m)
    out["end_der"] = out["end_der"].reshape(2, m)
    return out


# ------------------------------------------------------------ torch-facing wrappers

def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_ptr(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return t.data_ptr()


class Mesh:
    """Structured nx x ny x nz hexahedral mesh (vertices None: affine unit cube)."""

    def __init__(self, nx: int, ny: int, nz: int, vertices: Optional[np.ndarray] = None):
        self.shape = (nx, ny, nz)
        self.handle = dg_mesh_create(nx, ny, nz, vertices)

    @property
    def ncell(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            dg_mesh_destroy(h)
            self.handle = None


class Operator:
    """y = A x of the SIPG operator on a Mesh (see dg_operator_create)."""

    def __init__(self, mesh: Mesh, degree: int, *, quad_points: int = 0, c: float = 1.0, mu: float = 1.0,
                 theta: float = -1.0, penalty_mode: int = DG_PEN_CONFIG, penalty_alpha: float = 2.0,
                 dirichlet_mask: int = 0b111111, precision: int = DG_FP64, max_rhs: int = 1,
                 problem: int = DG_SCALAR, geometry: int = DG_GEOM_AUTO, degrees=None, quad=None):
        """degrees=(k_0, k_1, k_2): anisotropic degrees, quad=(m_0, m_1, m_2) their Gauss points
        (dg_operator_create_aniso; degree and quad_points unused)."""
        import torch
        self.mesh = mesh
        self.degree = degree
        self.precision = precision
        self.dtype = torch.float64 if precision == DG_FP64 else torch.float32
        self.max_rhs = max_rhs
        pen = dg_penalty(penalty_mode, 0, penalty_alpha)
        co = dg_coefficients(problem, precision, dirichlet_mask, max_rhs, geometry, 0, c, mu, theta)
        if degrees is not None:
            self.handle = dg_operator_create_aniso(mesh.handle, degrees, pen, co, quad)
        else:
            self.handle = dg_operator_create(mesh.handle, degree, quad_points, pen, co)
        self.ndofs = dg_operator_ndofs(self.handle)
        self._kappa = (None, None)

    def stats(self) -> dg_stats:
        return dg_operator_stats(self.handle)

    def autotune(self, nrhs: int = 1, stream=None) -> dict:
        return dg_operator_autotune(self.handle, nrhs, _stream_ptr(stream))

    def set_variant(self, variant: int, cells_per_block: int = 0, faces_per_block: int = 0):
        dg_operator_set_variant(self.handle, variant, cells_per_block, faces_per_block)

    def set_kappa(self, kappa_vol=None, kappa_face=None):
        """Per-quadrature-point kappa as device tensors of the operator's dtype (None = 1)."""
        pv = None if kappa_vol is None else _dev_ptr(kappa_vol, self.dtype, "kappa_vol")
        pf = None if kappa_face is None else _dev_ptr(kappa_face, self.dtype, "kappa_face")
        dg_operator_set_kappa(self.handle, pv, pf)
        self._kappa = (kappa_vol, kappa_face)  # keep alive while the operator reads them

    def apply(self, x, y=None, stream=None):
        """y = A x for x of shape [ndofs] or [nrhs, ndofs] (CUDA tensors)."""
        import torch
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if x.numel() != nrhs * self.ndofs:
            raise ValueError("x has the wrong size")
        if y is None:
            y = torch.empty_like(x)
        dg_apply(self.handle, _dev_ptr(x, self.dtype, "x"), _dev_ptr(y, self.dtype, "y"), nrhs, _stream_ptr(stream))
        return y

    def rhs(self, f_vol=None, g_face=None, stream=None):
        """F = (f, v) + theta (g, n.kappa grad v)_D + gamma (g, v)_D from point values (CUDA tensors)."""
        import torch
        F = torch.empty(self.ndofs, dtype=self.dtype, device="cuda")
        dg_rhs(self.handle, None if f_vol is None else _dev_ptr(f_vol, self.dtype, "f_vol"),
               None if g_face is None else _dev_ptr(g_face, self.dtype, "g_face"), F.data_ptr(), _stream_ptr(stream))
        return F

    def semilinear(self, w, beta, u0=None, stream=None):
        """u0 None: A w + beta (w^3, v); else A w + 3 beta (u0^2 w, v) (FP64 CUDA tensors)."""
        import torch
        if w.numel() != self.ndofs:
            raise ValueError("w has the wrong size")
        y = torch.empty_like(w)
        mode = DG_SEMILINEAR_RESIDUAL if u0 is None else DG_SEMILINEAR_JACOBIAN
        _check(lib().dg_apply_semilinear(self.handle, mode, float(beta),
                                         None if u0 is None else _dev_ptr(u0, self.dtype, "u0"),
                                         _dev_ptr(w, self.dtype, "w"), _dev_ptr(y, self.dtype, "y"),
                                         _stream_ptr(stream)), "dg_apply_semilinear")
        return y

    def block_jacobi(self, r, z=None, stream=None):
        """z = A_cc^-1 r per cell (cell-block Jacobi) for r of shape [ndofs] or [nrhs, ndofs]."""
        import torch
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        if r.numel() != nrhs * self.ndofs:
            raise ValueError("r has the wrong size")
        if z is None:
            z = torch.empty_like(r)
        dg_operator_block_jacobi(self.handle, _dev_ptr(r, self.dtype, "r"), _dev_ptr(z, self.dtype, "z"), nrhs,
                                 _stream_ptr(stream))
        return z

    def apply_host(self, x, y, stream=None):
        """y = A x through host buffers (numpy arrays or CPU tensors, ideally pinned)."""
        nrhs = 1 if x.ndim == 1 else x.shape[0]
        xp = x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
        yp = y.ctypes.data if isinstance(y, np.ndarray) else y.data_ptr()
        dg_apply_host(self.handle, xp, yp, nrhs, _stream_ptr(stream))
        return y

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            dg_operator_destroy(h)
            self.handle = None
