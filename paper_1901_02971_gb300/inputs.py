"""Seeded synthetic problem generators.

This module holds no part of the spaND method: it only builds SPD test
matrices (CSR, FP64), their optional vertex coordinates and right-hand
sides, shaped like the workloads the paper evaluates (Section 4: 2D/3D
elliptic problems discretised with 5- and 7-point stencils, variable
coefficients, algebraic SPD matrices without geometry).  Both the product
path (benchmarks, tests) and the FP64 oracle read their inputs from here.

Conventions
-----------
* Unknowns of a grid are ordered lexicographically, x fastest:
  ``i = x + n*y`` (2D), ``i = x + n*(y + n*z)`` (3D).
* Coordinates are the integer grid indices stored as float64 (exact).
* CSR arrays: ``rowptr`` int64 (N+1), ``colind`` int32 (sorted per row,
  diagonal included), ``vals`` float64.
* Variable-coefficient stencils (the elliptic operator of Section 4.1.1):
  the coefficient of the face between two cells is the harmonic mean of the
  two cell values; a face on the Dirichlet boundary uses the cell's own
  value and only adds to the diagonal.  No h^2 scaling.  With a == 1 this is
  the plain 5-/7-point Laplacian (diagonal 4 / 6, off-diagonals -1).
* Randomness: numpy ``Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class Problem:
    name: str
    n: int
    rowptr: np.ndarray  # int64 (n+1)
    colind: np.ndarray  # int32 (nnz)
    vals: np.ndarray    # float64 (nnz)
    coords: Optional[np.ndarray]  # float64 (n, dim) or None
    dim: int

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind.astype(np.int64), self.rowptr),
                             shape=(self.n, self.n))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _grid_coords(shape) -> np.ndarray:
    """Integer coordinates (x, y[, z]) of every cell of a grid given in numpy
    order (z, y, x) / (y, x), cells numbered x fastest; float64."""
    idx = np.indices(shape).reshape(len(shape), -1)[::-1]
    return np.ascontiguousarray(idx.T.astype(np.float64))


def _harm(a, b):
    return 2.0 * a * b / (a + b)


def _assemble(shape, cell: np.ndarray, name: str, axis_scale=None) -> Problem:
    """Variable-coefficient 5/7-point stencil on a grid with Dirichlet faces.

    ``cell`` has the grid shape in (z, y, x) / (y, x) order (numpy C order,
    so that ``cell.ravel()`` follows the unknown numbering).  ``axis_scale``
    (x, y[, z]) multiplies the face coefficients along each grid axis
    (anisotropy); default 1."""
    dim = len(shape)
    n_tot = int(np.prod(shape))
    a = cell.reshape(-1).astype(np.float64)
    ids = np.arange(n_tot, dtype=np.int64).reshape(cell.shape)
    diag = np.zeros(n_tot)
    rows, cols, vals = [], [], []
    for ax in range(dim):
        # numpy axis for grid dimension ax (x is the last numpy axis)
        nax = dim - 1 - ax
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[nax] = slice(0, -1)
        hi[nax] = slice(1, None)
        i0 = ids[tuple(lo)].ravel()
        i1 = ids[tuple(hi)].ravel()
        sc = 1.0 if axis_scale is None else float(axis_scale[ax])
        f = sc * _harm(a[i0], a[i1])
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [-f, -f]
        np.add.at(diag, i0, f)
        np.add.at(diag, i1, f)
        # Dirichlet faces on both ends of this axis
        first = [slice(None)] * dim
        last = [slice(None)] * dim
        first[nax] = 0
        last[nax] = -1
        for sl in (first, last):
            ib = ids[tuple(sl)].ravel()
            np.add.at(diag, ib, (1.0 if axis_scale is None else float(axis_scale[ax])) * a[ib])
    rows.append(np.arange(n_tot))
    cols.append(np.arange(n_tot))
    vals.append(diag)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n_tot + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Problem(name, n_tot, rowptr, c.astype(np.int32), v,
                   _grid_coords(shape), dim)


def laplacian_2d(n: int) -> Problem:
    """5-point Dirichlet Laplacian on an n x n grid (diag 4, off-diag -1)."""
    return _assemble((n, n), np.ones((n, n)), f"lapl2d_{n}")


def laplacian_3d(n: int) -> Problem:
    """7-point Dirichlet Laplacian on an n^3 grid (diag 6, off-diag -1)."""
    return _assemble((n, n, n), np.ones((n, n, n)), f"lapl3d_{n}")


def diffusion_3d(n: int, seed: int, block: int = 8, lo: float = -3.0,
                 hi: float = 3.0) -> Problem:
    """-div(a grad u) on n^3 cells; a = 10^u, u ~ U(lo, hi) i.i.d. per
    block^3 cell block (piecewise constant)."""
    nb = -(-n // block)
    u = rng(seed).uniform(lo, hi, size=(nb, nb, nb))
    cell = np.repeat(np.repeat(np.repeat(10.0 ** u, block, 0), block, 1), block, 2)
    return _assemble((n, n, n), cell[:n, :n, :n], f"diff3d_{n}_s{seed}")


def diffusion_2d(n: int, seed: int, sigma: float = 1.0) -> Problem:
    """-div(a grad u) on n^2 cells with log a ~ N(0, sigma^2) per cell."""
    cell = np.exp(sigma * rng(seed).standard_normal((n, n)))
    return _assemble((n, n), cell, f"diff2d_{n}_s{seed}")


def high_contrast_field(shape, rho: float, seed: int, sigma: float = 1.0) -> np.ndarray:
    """The quantized high-contrast coefficient field of the 2D experiments
    (Sec. 4.1): uniform (0, 1) noise per cell, smoothed by a Gaussian of
    standard deviation `sigma` cells (boundary: mirror reflection), then
    rho where the smoothed value is >= 0.5 and 1/rho elsewhere."""
    from scipy.ndimage import gaussian_filter
    a_hat = gaussian_filter(rng(seed).random(shape), sigma=sigma, mode="reflect")
    return np.where(a_hat >= 0.5, float(rho), 1.0 / float(rho))


def high_contrast_2d(n: int, rho: float, seed: int) -> Problem:
    """-div(a grad u) on n^2 cells with the quantized high-contrast field."""
    return _assemble((n, n), high_contrast_field((n, n), rho, seed), f"hc2d_{n}_r{rho:g}_s{seed}")


def high_contrast_3d(n: int, rho: float, seed: int) -> Problem:
    """-div(a grad u) on n^3 cells with the quantized high-contrast field."""
    return _assemble((n, n, n), high_contrast_field((n, n, n), rho, seed), f"hc3d_{n}_r{rho:g}_s{seed}")


def extruded_3d(nx: int, ny: int, nz: int, seed: int, aniso: float = 100.0) -> Problem:
    """Thin extruded 3D problem (stand-in for the ice-sheet runs of Sec. 4):
    7-point -div(a grad u) on nx x ny x nz cells, nz small, with a background
    field varying over six decades in the plane, a = 10^(3 s(x, y)), s a
    Gaussian-smoothed (sigma = 4 cells) uniform noise rescaled to [-1, 1] and
    constant along z, and vertical faces `aniso` times stronger (thin
    layers).  Coordinates are the (x, y) of every cell only, so that the
    geometric separator partitions the plane and extrudes the partition in z.
    """
    from scipy.ndimage import gaussian_filter
    s = gaussian_filter(rng(seed).random((ny, nx)), sigma=4.0, mode="reflect")
    s = 2.0 * (s - s.min()) / max(s.max() - s.min(), 1e-300) - 1.0
    cell = np.broadcast_to(10.0 ** (3.0 * s), (nz, ny, nx)).copy()
    p = _assemble((nz, ny, nx), cell, f"extr_{nx}x{ny}x{nz}_s{seed}", axis_scale=(1.0, 1.0, aniso))
    xy = _grid_coords((nz, ny, nx))[:, :2].copy()
    return Problem(p.name, p.n, p.rowptr, p.colind, p.vals, xy, 2)


def knn_laplacian(npts: int, k: int, seed: int, shift: float = 1e-4) -> Problem:
    """Graph Laplacian of the symmetrised k-NN graph of uniform points in the
    unit cube, weights exp(-d^2/h^2) with h the mean k-th neighbour distance,
    plus shift*I.  Returned without coordinates (purely algebraic input)."""
    from scipy.spatial import cKDTree
    pts = rng(seed).random((npts, 3))
    tree = cKDTree(pts)
    d, j = tree.query(pts, k=k + 1)
    d, j = d[:, 1:], j[:, 1:]
    h = float(np.mean(d[:, -1]))
    i = np.repeat(np.arange(npts), k)
    j = j.ravel()
    w = np.exp(-(d.ravel() ** 2) / h ** 2)
    # symmetrise by union: keep each unordered pair once (max weight is the
    # same value from either side since the weight depends only on distance)
    a = np.minimum(i, j)
    b = np.maximum(i, j)
    key = a.astype(np.int64) * npts + b
    key, first = np.unique(key, return_index=True)
    a, b, w = a[first], b[first], w[first]
    rows = np.concatenate([a, b, np.arange(npts)])
    cols = np.concatenate([b, a, np.arange(npts)])
    deg = np.zeros(npts)
    np.add.at(deg, a, w)
    np.add.at(deg, b, w)
    vals = np.concatenate([-w, -w, deg + shift])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(npts + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Problem(f"knn_{npts}_k{k}_s{seed}", npts, rowptr,
                   cols.astype(np.int32), vals, None, 3)


def batch_diffusion_2d(i: int):
    """Problem i (0..31) of the batch of independent 2D diffusion systems:
    n_i = 128 + floor(384 i / 31) cells per side, log a ~ N(0, 1) per cell
    (seed 4 + i), x* ~ N(0, 1) (seed 100 + i), b = A x*, and the level count
    L_i = round(log2(N_i / 32)) + 1.  Returns (problem, x*, b, L_i)."""
    n = 128 + (384 * i) // 31
    p = diffusion_2d(n, 4 + i)
    xs = rng(100 + i).standard_normal(p.n)
    b = p.to_scipy() @ xs
    return p, xs, b, int(round(np.log2(p.n / 32))) + 1


def sketch_gaussian(seed: int, step: int, cluster: int, m: int, ell: int) -> np.ndarray:
    """Gaussian test matrix (m x ell) with i.i.d. N(0, 1) entries for the
    randomized compression of one interface: drawn column by column from
    PCG64 seeded by the triple (seed, step, cluster), so that the first j
    columns are the same for every ell >= j (a sketch can grow without
    redrawing)."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, step, cluster])))
    return g.standard_normal((ell, m)).T


def rhs(n: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1), seeded."""
    return rng(seed).standard_normal(n)


def by_name(name: str) -> Problem:
    """Named workloads used by the tests and the benchmark."""
    if name == "lapl2d_64":
        return laplacian_2d(64)
    if name == "lapl3d_64":
        return laplacian_3d(64)
    if name.startswith("lapl2d_"):
        return laplacian_2d(int(name.split("_")[1]))
    if name.startswith("lapl3d_"):
        return laplacian_3d(int(name.split("_")[1]))
    raise KeyError(name)
