"""ctypes shim over the C oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package. It evaluates the SIPG-DG bilinear forms of arXiv 1812.08075
(Eq. diffreac_weak, Sec. 5.2; Eq. stokes_weak, Sec. 5.3) by full basis evaluation at
Gauss points; see ``oracle.h`` for the readings of the paper it fixes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP) into _build/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall", "-Wno-unknown-pragmas",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("k", ctypes.c_int32), ("m", ctypes.c_int32), ("pen_mode", ctypes.c_int32),
        ("dirichlet_mask", ctypes.c_int32), ("problem", ctypes.c_int32),
        ("c", ctypes.c_double), ("mu", ctypes.c_double), ("theta", ctypes.c_double),
        ("pen_alpha", ctypes.c_double),
        ("vertices", ctypes.c_void_p), ("kappa_vol", ctypes.c_void_p), ("kappa_face", ctypes.c_void_p),
        ("kaxis", ctypes.c_int32 * 3), ("maxis", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Problem)
        dp = ctypes.c_void_p
        lib.oracle_gauss_rule.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_gll_nodes.argtypes = [ctypes.c_int, dp]
        lib.oracle_ndofs.argtypes = [P]
        lib.oracle_ndofs.restype = ctypes.c_int64
        lib.oracle_apply.argtypes = [P, ctypes.c_int, dp, dp]
        lib.oracle_apply_cells.argtypes = [P, ctypes.c_int, dp, ctypes.c_int64, dp, dp, ctypes.c_int]
        lib.oracle_dkappa.argtypes = [P, dp, dp, dp, dp]
        lib.oracle_rhs.argtypes = [P, dp, dp, dp]
        lib.oracle_semilinear.argtypes = [P, ctypes.c_double, ctypes.c_int, dp, dp, dp]
        lib.oracle_assemble_coo.argtypes = [P, ctypes.c_int64, dp, dp, dp]
        lib.oracle_assemble_coo.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def gauss_rule(m: int):
    """m-point Gauss-Legendre rule on [0,1] (nodes ascending, weights)."""
    lib = _load()
    s = np.zeros(m)
    w = np.zeros(m)
    if lib.oracle_gauss_rule(m, _ptr(s), _ptr(w)):
        raise ValueError("bad m")
    return s, w


def gll_nodes(k: int):
    """k+1 Gauss-Lobatto-Legendre points on [0,1]."""
    lib = _load()
    z = np.zeros(k + 1)
    if lib.oracle_gll_nodes(k, _ptr(z)):
        raise ValueError("bad k")
    return z


@dataclass
class Problem:
    """Parameters of one operator (field meanings as in ``oracle.h``)."""
    nx: int
    ny: int
    nz: int
    k: int
    m: Optional[int] = None
    problem: str = "scalar"          # "scalar" | "stokes"
    c: float = 1.0
    mu: float = 1.0
    theta: float = -1.0
    pen_mode: int = 0
    pen_alpha: float = 2.0
    dirichlet_mask: int = 0b111111
    vertices: Optional[np.ndarray] = None
    kappa_vol: Optional[np.ndarray] = None
    kappa_face: Optional[np.ndarray] = None
    degrees: Optional[tuple] = None  # anisotropic (k_0, k_1, k_2): scalar problem
    quad: Optional[tuple] = None     # with degrees: Gauss points (m_0, m_1, m_2), None = k_a + 1

    def __post_init__(self):
        if self.m is None:
            self.m = self.k + 1

    @property
    def local_size(self) -> int:
        if self.degrees is not None:
            return int(np.prod([d + 1 for d in self.degrees]))
        return self.ndofs() // self.ncell

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def _struct(self):
        keep = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data

        s = _Problem(self.nx, self.ny, self.nz, self.k, self.m, self.pen_mode, self.dirichlet_mask,
                     0 if self.problem == "scalar" else 1, self.c, self.mu, self.theta, self.pen_alpha,
                     arr(self.vertices), arr(self.kappa_vol), arr(self.kappa_face),
                     (ctypes.c_int32 * 3)(*(self.degrees or (0, 0, 0))),
                     (ctypes.c_int32 * 3)(*(self.quad or (0, 0, 0))), 0)
        return s, keep

    def ndofs(self) -> int:
        s, _ = self._struct()
        n = _load().oracle_ndofs(ctypes.byref(s))
        if n < 0:
            raise ValueError("invalid problem")
        return int(n)

    def apply(self, x: np.ndarray, transpose: bool = False) -> np.ndarray:
        """y = A x (or A^T x), element-wise over cells and faces."""
        s, keep = self._struct()
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.ndofs())
        if x.size != y.size:
            raise ValueError("x has the wrong size")
        if _load().oracle_apply(ctypes.byref(s), int(transpose), _ptr(x), _ptr(y)):
            raise RuntimeError("oracle_apply failed")
        return y

    def apply_cells(self, x: np.ndarray, cells: np.ndarray, transpose: bool = False,
                    nthreads: int = 0) -> np.ndarray:
        """(A x) restricted to the listed cells, shape [len(cells), local size]."""
        s, keep = self._struct()
        x = np.ascontiguousarray(x, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        loc = self.ndofs() // self.ncell
        y = np.zeros((cells.size, loc))
        if _load().oracle_apply_cells(ctypes.byref(s), int(transpose), _ptr(x), cells.size, _ptr(cells),
                                      _ptr(y), int(nthreads)):
            raise RuntimeError("oracle_apply_cells failed")
        return y

    def dkappa(self, x: np.ndarray, r: np.ndarray):
        """(dL/dkappa_vol, dL/dkappa_face) for L = 0.5||A x - b||^2 with r = A x - b."""
        s, keep = self._struct()
        x = np.ascontiguousarray(x, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        dv = np.zeros(self.ncell * self.m ** 3)
        df = np.zeros(self.ncell * 6 * self.m ** 2)
        if _load().oracle_dkappa(ctypes.byref(s), _ptr(x), _ptr(r), _ptr(dv), _ptr(df)):
            raise RuntimeError("oracle_dkappa failed")
        return dv, df

    def rhs(self, f_vol=None, g_face=None) -> np.ndarray:
        """F = (f, v) + theta (g, n.kappa grad v)_D + gamma (g, v)_D (data terms, r = A u - F)."""
        s, keep = self._struct()
        fv = None if f_vol is None else np.ascontiguousarray(f_vol, dtype=np.float64)
        gf = None if g_face is None else np.ascontiguousarray(g_face, dtype=np.float64)
        F = np.zeros(self.ndofs())
        if _load().oracle_rhs(ctypes.byref(s), _ptr(fv), _ptr(gf), _ptr(F)):
            raise RuntimeError("oracle_rhs failed")
        return F

    def semilinear(self, w: np.ndarray, beta: float, u0: Optional[np.ndarray] = None) -> np.ndarray:
        """u0 None: A w + beta (w^3, v) (residual operator); else A w + 3 beta (u0^2 w, v)
        (its Jacobian action at u0)."""
        s, keep = self._struct()
        w = np.ascontiguousarray(w, dtype=np.float64)
        u = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
        y = np.zeros(self.ndofs())
        if _load().oracle_semilinear(ctypes.byref(s), float(beta), 0 if u is None else 1, _ptr(u), _ptr(w), _ptr(y)):
            raise RuntimeError("oracle_semilinear failed")
        return y

    def block_jacobi(self, r: np.ndarray) -> np.ndarray:
        """z with A_cc z_c = r_c for every cell c, A_cc the cell's diagonal block of the
        assembled matrix (cell-block Jacobi; dense solves, small meshes only)."""
        A = self.assemble()
        loc = self.ndofs() // self.ncell
        r = np.asarray(r, dtype=np.float64)
        z = np.empty_like(r)
        for c in range(self.ncell):
            sl = slice(c * loc, (c + 1) * loc)
            z[sl] = np.linalg.solve(A[sl, sl].toarray(), r[sl])
        return z

    def assemble(self):
        """Sparse matrix A (scipy CSR) from the local cell and face matrices."""
        import scipy.sparse as sp
        s, keep = self._struct()
        lib = _load()
        need = lib.oracle_assemble_coo(ctypes.byref(s), 0, None, None, None)
        if need < -(1 << 60):
            raise RuntimeError("oracle_assemble_coo failed")
        cap = -need if need < 0 else 1
        rows = np.zeros(cap, dtype=np.int64)
        cols = np.zeros(cap, dtype=np.int64)
        vals = np.zeros(cap)
        cnt = lib.oracle_assemble_coo(ctypes.byref(s), cap, _ptr(rows), _ptr(cols), _ptr(vals))
        if cnt < 0:
            raise RuntimeError("oracle_assemble_coo failed")
        n = self.ndofs()
        return sp.coo_matrix((vals[:cnt], (rows[:cnt], cols[:cnt])), shape=(n, n)).tocsr()
