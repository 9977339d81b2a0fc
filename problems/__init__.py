"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver: it only produces sparse
matrices (CSR, natural grid numbering) and right-hand sides.  Both the CPU
oracle and the CUDA library consume what it produces, so neither side has
to import the other.

Workloads follow the PDE benchmarks of Section 6.1 of the paper (Poisson on
regular 2D/3D grids with the standard 5-/7-point stencils and homogeneous
Dirichlet conditions), plus the variants used by the scaled configurations:
an upwinded 2D convection-diffusion operator and a shifted 3D Laplacian.

Natural numbering: vertex (x, y, z) of an nx*ny*nz grid has index
x + nx*(y + ny*z).  Column indices are ascending inside every row.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_dims",
    "grid_poisson",
    "grid_convdiff2d",
    "grid_shifted_laplacian3d",
    "grid_anisotropic_grf",
    "gaussian_random_field",
    "rhs_uniform",
    "block_diag",
    "batch_convdiff2d",
    "CSR",
]


class CSR:
    """A square sparse matrix in compressed-sparse-row form (0-based)."""

    def __init__(self, n, rowptr, colind, values):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.values = np.ascontiguousarray(values, dtype=np.float64)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.values, self.colind, self.rowptr), shape=(self.n, self.n))


def grid_dims(dims):
    """Normalise (nx,), (nx, ny) or (nx, ny, nz) to a 3-tuple."""
    d = [int(v) for v in dims]
    while len(d) < 3:
        d.append(1)
    if any(v < 1 for v in d):
        raise ValueError("grid sides must be positive")
    return tuple(d)


def _stencil_pattern(dims, offsets):
    nx, ny, nz = grid_dims(dims)
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    rows, cols, kinds = [], [], []
    for k, (dx, dy, dz) in enumerate(offsets):
        xx, yy, zz = x + dx, y + dy, z + dz
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        rows.append(idx[ok])
        cols.append((xx + nx * (yy + ny * zz))[ok])
        kinds.append(np.full(int(ok.sum()), k, dtype=np.int64))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    kinds = np.concatenate(kinds)
    order = np.lexsort((cols, rows))
    rows, cols, kinds = rows[order], cols[order], kinds[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return n, rowptr, cols, kinds, (x, y, z)


def _offsets(dim3, stencil):
    if stencil in (5, 7):
        offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
        if stencil == 7:
            offs += [(0, 0, -1), (0, 0, 1)]
        return offs
    raise ValueError("stencil must be 5 (2D) or 7 (3D)")


def grid_poisson(dims, stencil=None, scale=1.0):
    """Standard 5-point (2D) or 7-point (3D) Laplacian, Dirichlet boundary.

    Diagonal 4 (2D) or 6 (3D), off-diagonal -1 towards every grid
    neighbour, times ``scale`` (pass (k+1)**2 for the h^-2 scaling of a
    k-point-per-side unit-square grid).  Section 6.1 of the paper.
    """
    nx, ny, nz = grid_dims(dims)
    if stencil is None:
        stencil = 7 if nz > 1 else 5
    offs = _offsets(3, stencil)
    n, rowptr, cols, kinds, _ = _stencil_pattern((nx, ny, nz), offs)
    diag = 2.0 * (len(offs) - 1) / 2.0
    vals = np.where(kinds == 0, diag, -1.0) * float(scale)
    return CSR(n, rowptr, cols, vals)


def grid_convdiff2d(side, vx, vy, nu=1.0):
    """Upwinded 5-point convection-diffusion -nu*Lap(u) + v.grad(u) on a
    side x side interior grid of the unit square, h = 1/(side+1), constant
    velocity (vx, vy).  Diagonal 4nu/h^2 + |vx|/h + |vy|/h; the neighbour on
    the upwind side of each axis gets -nu/h^2 - |v|/h, the other -nu/h^2.
    """
    h = 1.0 / (side + 1)
    offs = _offsets(3, 5)
    n, rowptr, cols, kinds, _ = _stencil_pattern((side, side, 1), offs)
    dif = nu / h ** 2
    vals = np.empty(len(cols))
    vals[kinds == 0] = 4 * dif + abs(vx) / h + abs(vy) / h
    # kinds: 1 = x-1, 2 = x+1, 3 = y-1, 4 = y+1
    vals[kinds == 1] = -dif - max(vx, 0.0) / h
    vals[kinds == 2] = -dif - max(-vx, 0.0) / h
    vals[kinds == 3] = -dif - max(vy, 0.0) / h
    vals[kinds == 4] = -dif - max(-vy, 0.0) / h
    return CSR(n, rowptr, cols, vals)


def grid_shifted_laplacian3d(side, sigma):
    """-Lap(u) + sigma*u, 7-point, unscaled stencil, sigma per cell (n values)."""
    offs = _offsets(3, 7)
    n, rowptr, cols, kinds, _ = _stencil_pattern((side, side, side), offs)
    sigma = np.asarray(sigma, dtype=np.float64).reshape(-1)
    if sigma.size != n:
        raise ValueError("sigma needs one value per cell")
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    vals = np.where(kinds == 0, 6.0 + sigma[rows], -1.0)
    return CSR(n, rowptr, cols, vals)


def gaussian_random_field(side, corr_len=8.0, sigma=1.0, seed=0):
    """A seeded stationary Gaussian random field on side^3 cells: white noise
    filtered in Fourier space by a Gaussian kernel of correlation length
    corr_len cells (periodic), shifted and scaled to mean 0 and standard
    deviation sigma.  Returned in natural order (x fastest)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((side, side, side))
    k = 2.0 * np.pi * np.fft.fftfreq(side)
    kr = 2.0 * np.pi * np.fft.rfftfreq(side)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    g = np.fft.irfftn(np.fft.rfftn(w) * np.exp(-0.5 * k2 * corr_len ** 2), s=w.shape)
    g = (g - g.mean()) / max(g.std(), 1e-300) * sigma
    # array axes (a, b, c) -> grid (z, y, x): natural index x + side (y + side z)
    return np.ascontiguousarray(g).reshape(-1)


def grid_anisotropic_grf(side, corr_len=8.0, sigma=1.0, aniso=(1.0, 1.0, 10.0), seed=0):
    """-div(K grad u) on the side^3 interior grid, 7-point finite volumes,
    homogeneous Dirichlet conditions: cell coefficient kappa = exp(g) with g
    a Gaussian random field (gaussian_random_field), the face between two
    cells the harmonic mean of their coefficients times the anisotropy factor
    of the face's axis (x, y, z), a boundary face the cell's own coefficient
    times that factor.  Symmetric positive definite; unscaled (h = 1)."""
    offs = _offsets(3, 7)
    n, rowptr, cols, kinds, _ = _stencil_pattern((side, side, side), offs)
    kappa = np.exp(gaussian_random_field(side, corr_len, sigma, seed))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    axis_of = np.array([-1, 0, 0, 1, 1, 2, 2])  # offsets: self, -x, +x, -y, +y, -z, +z
    a = np.asarray(aniso, dtype=np.float64)
    off = kinds != 0
    ki, kj = kappa[rows[off]], kappa[cols[off]]
    face = 2.0 * ki * kj / (ki + kj) * a[axis_of[kinds[off]]]
    vals = np.zeros(len(cols))
    vals[off] = -face
    # diagonal: all six faces of the cell (interior faces from the row's
    # off-diagonal entries, boundary faces from the cell's own coefficient)
    diag = np.zeros(n)
    np.add.at(diag, rows[off], face)
    idx = np.arange(n)
    x, y, z = idx % side, (idx // side) % side, idx // (side * side)
    nb = [(x == 0).astype(float) + (x == side - 1), (y == 0).astype(float) + (y == side - 1),
          (z == 0).astype(float) + (z == side - 1)]
    for ax in range(3):
        diag += nb[ax] * kappa * a[ax]
    vals[kinds == 0] = diag[rows[kinds == 0]]
    return CSR(n, rowptr, cols, vals)


def rhs_uniform(n, nrhs=1, seed=1):
    """Right-hand sides uniform on [-1, 1] from numpy's default_rng(seed),
    returned column-major as an (n, nrhs) float64 array."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=(nrhs, n)).T
    return np.asfortranarray(b)


def block_diag(mats):
    """The block-diagonal matrix of a list of CSR matrices (system s takes the
    natural indices after those of systems 0..s-1)."""
    n = sum(m.n for m in mats)
    rowptr = [np.zeros(1, dtype=np.int64)]
    cols, vals = [], []
    r0 = c0 = 0
    for m in mats:
        rowptr.append(m.rowptr[1:].astype(np.int64) + r0)
        cols.append(m.colind.astype(np.int64) + c0)
        vals.append(m.values)
        r0 += m.nnz
        c0 += m.n
    return CSR(n, np.concatenate(rowptr), np.concatenate(cols), np.concatenate(vals))


def batch_convdiff2d(nsys, side_lo=32, side_hi=256, vmax=50.0, nu=1.0, seed=0):
    """nsys independent upwinded 2D convection-diffusion systems
    (``grid_convdiff2d``): grid sides uniform on {side_lo..side_hi}, one
    constant velocity per system with components uniform on [-vmax, vmax],
    all drawn from one seeded stream.  Returns (sides, velocities, the
    block-diagonal CSR)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=nsys)
    vel = rng.uniform(-vmax, vmax, size=(nsys, 2))
    mats = [grid_convdiff2d(int(k), float(v[0]), float(v[1]), nu) for k, v in zip(sides, vel)]
    return [int(k) for k in sides], vel, block_diag(mats)
