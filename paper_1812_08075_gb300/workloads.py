"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only draws numbers and lays out the structured hexahedral mesh; it holds
none of the discretisation's arithmetic (no basis, quadrature, geometry or operator).
Both sides receive the same arrays from here, so a parity test compares the two
implementations on identical inputs.

Conventions (the paper's structured cuboid setting, Sec. 2.1):
  * cells are numbered lexicographically c = cx + nx*(cy + ny*cz);
  * mesh vertices are numbered v = i + (nx+1)*(j + (ny+1)*l), coordinates [nv, 3];
  * the scalar DOF vector is cell-major, [ncell][(k+1)^3];
  * per-quadrature-point coefficients are [ncell][m^3] (volume) and
    [ncell][6][m^2] (each cell's own side of its six faces, order -x,+x,-y,+y,-z,+z).
"""
from __future__ import annotations

import numpy as np


def unit_cube_vertices(nx: int, ny: int, nz: int) -> np.ndarray:
    """Vertices of the uniform nx*ny*nz lattice on [0,1]^3, shape [(nx+1)(ny+1)(nz+1), 3]."""
    gx = np.arange(nx + 1, dtype=np.float64) / nx
    gy = np.arange(ny + 1, dtype=np.float64) / ny
    gz = np.arange(nz + 1, dtype=np.float64) / nz
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).copy()


def perturbed_vertices(nx: int, ny: int, nz: int, amplitude: float = 0.1, seed: int = 1) -> np.ndarray:
    """Unit-cube lattice whose interior vertices are moved independently in each
    coordinate by U[-amplitude*h_a, +amplitude*h_a] (h_a = 1/n_a).

    One draw of shape [nv, 3] is taken from ``np.random.default_rng(seed)`` in vertex
    order; boundary vertices discard their draw, so the domain stays the unit cube and
    every boundary face stays planar.
    """
    v = unit_cube_vertices(nx, ny, nz)
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.0, 1.0, size=v.shape)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    i = np.arange(v.shape[0])
    ix = i % (nx + 1)
    iy = (i // (nx + 1)) % (ny + 1)
    iz = i // ((nx + 1) * (ny + 1))
    interior = (ix > 0) & (ix < nx) & (iy > 0) & (iy < ny) & (iz > 0) & (iz < nz)
    v[interior] += amplitude * d[interior] * h[None, :]
    return v


def uniform_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """x ~ U[-1, 1]^n from ``np.random.default_rng(seed)``."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n).astype(dtype)


def lognormal_kappa(ncell: int, m: int, seed: int = 2, sigma: float = 0.5):
    """Per-quadrature-point diffusion coefficient with log(kappa) ~ N(0, sigma^2).

    One draw of n_vol + n_face normals (volume values first, then face values, each in
    its flattened array order) from ``np.random.default_rng(seed)``.
    Returns (kappa_vol [ncell*m^3], kappa_face [ncell*6*m^2]).
    """
    nv = ncell * m ** 3
    nf = ncell * 6 * m * m
    g = np.random.default_rng(seed).normal(0.0, sigma, size=nv + nf)
    k = np.exp(g)
    return k[:nv].copy(), k[nv:].copy()


def lognormal_kappa_aniso(ncell: int, quad, seed: int = 2, sigma: float = 0.5):
    """lognormal_kappa for per-direction point counts quad = (m0, m1, m2): kappa_vol
    [ncell * m0 m1 m2] and kappa_face [ncell * 2 (m1 m2 + m0 m2 + m0 m1)] (six faces, each
    with the points of its two tangential directions), one draw, volume values first."""
    m0, m1, m2 = quad
    nv = ncell * m0 * m1 * m2
    nf = ncell * 2 * (m1 * m2 + m0 * m2 + m0 * m1)
    k = np.exp(np.random.default_rng(seed).normal(0.0, sigma, size=nv + nf))
    return k[:nv].copy(), k[nv:].copy()


def sin_product_source(nx: int, ny: int, nz: int, nodes) -> np.ndarray:
    """The smooth source f = sin(pi x) sin(pi y) sin(pi z) of the mixed-precision solve,
    evaluated at the volume points of the uniform unit-cube lattice: cell c's point q is
    ((cx + s_q0)/nx, (cy + s_q1)/ny, (cz + s_q2)/nz) for the caller's 1D points s on [0,1]
    (its own quadrature nodes). Layout [ncell][m^3], q = q0 + m (q1 + m q2)."""
    s = np.asarray(nodes, dtype=np.float64)
    m = s.size
    gx = np.sin(np.pi * (np.arange(nx)[:, None] + s[None, :]) / nx)
    gy = np.sin(np.pi * (np.arange(ny)[:, None] + s[None, :]) / ny)
    gz = np.sin(np.pi * (np.arange(nz)[:, None] + s[None, :]) / nz)
    f = (gz.reshape(nz, 1, 1, m, 1, 1) * gy.reshape(1, ny, 1, 1, m, 1)) * gx.reshape(1, 1, nx, 1, 1, m)
    return np.ascontiguousarray(f).reshape(-1)


def projected_rhs(load, seeds, dtype=np.float64) -> np.ndarray:
    """Right-hand sides b_s = l / max|l| + eta_s of the mixed-precision solve, with l the
    load vector (f, phi_i) of ``sin_product_source`` (integrated by the caller's own
    quadrature) and eta_s ~ U[-1,1] from seed s. Shape [len(seeds), l.size]."""
    l = np.asarray(load, dtype=np.float64)
    l = l / np.abs(l).max()
    out = np.empty((len(seeds), l.size), dtype=dtype)
    for i, sd in enumerate(seeds):
        out[i] = l + uniform_vector(l.size, sd)
    return out


def cell_centre_sin_source(nx: int, ny: int, nz: int, ndof_per_cell: int) -> np.ndarray:
    """A smooth test vector: sin(pi x) sin(pi y) sin(pi z) at each cell's centre, repeated
    over the cell's DOFs (the unit-cube lattice, no basis or quadrature involved)."""
    cx = (np.arange(nx) + 0.5) / nx
    cy = (np.arange(ny) + 0.5) / ny
    cz = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    s = (np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)).ravel()
    return np.repeat(s, ndof_per_cell)


def refinement_rhs(nx: int, ny: int, nz: int, ndof_per_cell: int, seeds, dtype=np.float64) -> np.ndarray:
    """Smooth-plus-noise test vectors b_s = v / max|v| + eta_s with v the cell-centre
    sin-product above and eta_s ~ U[-1,1] from seed s (generic solver inputs that need
    no quadrature). Shape [len(seeds), ncell*ndof_per_cell]."""
    return projected_rhs(cell_centre_sin_source(nx, ny, nz, ndof_per_cell), seeds, dtype)


def sample_cells(ncell: int, count: int, seed: int = 7) -> np.ndarray:
    """A sorted, duplicate-free random sample of cell indices that always contains the
    first and last cell (corner cells touch three boundary faces)."""
    rng = np.random.default_rng(seed)
    count = min(count, ncell)
    pick = rng.choice(ncell, size=count, replace=False)
    pick = np.unique(np.concatenate([pick, [0, ncell - 1]]))
    return pick.astype(np.int64)
