"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the SAIT method.  It only builds the
coefficient matrices of the model PDE problems (finite-difference stencils),
right-hand sides and random triangular test matrices, as plain numpy CSR
arrays (int32 row pointers and column indices, float64 values, columns sorted
ascending within each row, the diagonal always stored).

The paper's own workload is the 7-point finite-difference Laplacian on the
unit cube with a 102^3 mesh, i.e. 100^3 interior unknowns and homogeneous
Dirichlet boundary conditions (Section 4, equations Lap_00 and A_u_f).  The
other generators are the larger synthetic PDE problems the GPU path is
measured on (3D convection-diffusion, log-normal diffusion, anisotropic 2D
Poisson); every matrix is scaled by h^2 so that the stencil weights are O(1).

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), which
gives the same stream on every platform numpy supports.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "poisson2d", "laplace3d", "convdiff3d", "varcoef3d", "aniso2d",
    "aniso2d_batch_params", "random_triangular", "uniform", "from_dense",
    "SEED_BASE",
]

# Seeds of the synthetic workloads are SEED_BASE + a small workload index.
SEED_BASE = 2106128360


@dataclass
class CSR:
    """Square sparse matrix in CSR form (int32 indices, float64 values)."""

    n: int
    rp: np.ndarray   # int32[n+1]
    ci: np.ndarray   # int32[nnz], ascending within each row
    va: np.ndarray   # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rp[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rp))
        d[rows, self.ci] = self.va
        return d

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.va, self.ci, self.rp), shape=(self.n, self.n))

    def row(self, i: int):
        a, b = int(self.rp[i]), int(self.rp[i + 1])
        return self.ci[a:b], self.va[a:b]


def from_dense(d: np.ndarray, keep_zero_diag: bool = True) -> CSR:
    """CSR of a dense square matrix; structural nonzeros are the nonzero entries."""
    n = d.shape[0]
    mask = d != 0
    if keep_zero_diag:
        mask[np.arange(n), np.arange(n)] = True
    rows, cols = np.nonzero(mask)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return CSR(n, rp, cols.astype(np.int32), d[rows, cols].astype(np.float64))


def _assemble(cols: np.ndarray, vals: np.ndarray, valid: np.ndarray) -> CSR:
    """Rows of (cols, vals) candidates in ascending column order, masked by valid."""
    n = cols.shape[0]
    counts = valid.sum(axis=1)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(counts)
    ci = cols[valid].astype(np.int32)
    va = vals[valid].astype(np.float64)
    return CSR(n, rp.astype(np.int32), ci, va)


def _stencil3d(N: int, coef: dict) -> CSR:
    """7-point stencil on an N^3 grid, natural ordering idx = x + N*y + N^2*z.

    ``coef`` maps offsets (dx,dy,dz) to an array (or scalar) of weights per row.
    """
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    order = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.empty((n, 7), dtype=np.float64)
    valid = np.empty((n, 7), dtype=bool)
    for c, (dx, dy, dz) in enumerate(order):
        cols[:, c] = idx + dx + N * dy + N * N * dz
        valid[:, c] = ((x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N)
                       & (z + dz >= 0) & (z + dz < N))
        vals[:, c] = coef[(dx, dy, dz)]
    return _assemble(cols, vals, valid)


def poisson2d(g: int) -> CSR:
    """5-point Poisson on a g x g interior grid (h^2-scaled: 4 on the diagonal, -1 off)."""
    n = g * g
    idx = np.arange(n, dtype=np.int64)
    x = idx % g
    y = idx // g
    cols = np.stack([idx - g, idx - 1, idx, idx + 1, idx + g], axis=1)
    valid = np.stack([y > 0, x > 0, np.ones(n, bool), x < g - 1, y < g - 1], axis=1)
    vals = np.tile(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (n, 1))
    return _assemble(cols, vals, valid)


def aniso2d(g: int, eps: float) -> CSR:
    """5-point -eps*u_xx - u_yy on a g x g interior grid (h^2-scaled)."""
    n = g * g
    idx = np.arange(n, dtype=np.int64)
    x = idx % g
    y = idx // g
    cols = np.stack([idx - g, idx - 1, idx, idx + 1, idx + g], axis=1)
    valid = np.stack([y > 0, x > 0, np.ones(n, bool), x < g - 1, y < g - 1], axis=1)
    vals = np.tile(np.array([-1.0, -eps, 2.0 * eps + 2.0, -eps, -1.0]), (n, 1))
    return _assemble(cols, vals, valid)


def aniso2d_batch_params(count: int, seed: int, smin: int = 16, smax: int = 256):
    """Grid sides s ~ U{smin..smax} and anisotropies eps = 10^U[-3,0] for a batch."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(smin, smax + 1, size=count)
    eps = 10.0 ** rng.uniform(-3.0, 0.0, size=count)
    return sides.astype(np.int64), eps


def laplace3d(N: int) -> CSR:
    """7-point Laplacian on an N^3 interior grid (h^2-scaled: 6 on the diagonal, -1 off).

    N = 100 is the paper's test problem (a 102^3 mesh including the boundary).
    """
    coef = {o: -1.0 for o in [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]}
    coef[(0, 0, 0)] = 6.0
    return _stencil3d(N, coef)


def convdiff3d(N: int, beta=(1.0, 0.5, 0.25), peclet: float = 0.5) -> CSR:
    """7-point central-difference -Lap(u) + beta.grad(u) on an N^3 grid (h^2-scaled).

    The convection vector is scaled so that the cell Peclet number beta_d*h/2 of
    its largest component equals ``peclet``.  Neighbour weights are -1 + Pe_d
    downstream (+d) and -1 - Pe_d upstream (-d); the diagonal is 6.  For
    Pe_d < 1 the matrix is a nonsymmetric M-matrix.
    """
    b = np.asarray(beta, dtype=np.float64)
    pe = peclet * b / np.max(np.abs(b))
    coef = {
        (0, 0, 0): 6.0,
        (1, 0, 0): -1.0 + pe[0], (-1, 0, 0): -1.0 - pe[0],
        (0, 1, 0): -1.0 + pe[1], (0, -1, 0): -1.0 - pe[1],
        (0, 0, 1): -1.0 + pe[2], (0, 0, -1): -1.0 - pe[2],
    }
    return _stencil3d(N, coef)


def varcoef3d(N: int, sigma: float, seed: int) -> CSR:
    """7-point -div(kappa grad u) on an N^3 grid with log-normal cell coefficients.

    kappa_cell = exp(sigma * g), g ~ N(0,1) i.i.d. per cell.  The coefficient of an
    interior face is the harmonic mean of its two cells; a boundary face uses
    the cell's own kappa (Dirichlet value at distance h).  Symmetric M-matrix.
    """
    rng = np.random.default_rng(seed)
    kap = np.exp(sigma * rng.standard_normal(N ** 3))
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    order = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.zeros((n, 7), dtype=np.float64)
    valid = np.empty((n, 7), dtype=bool)
    diag = np.zeros(n)
    for c, (dx, dy, dz) in enumerate(order):
        if (dx, dy, dz) == (0, 0, 0):
            cols[:, c] = idx
            valid[:, c] = True
            continue
        nb = idx + dx + N * dy + N * N * dz
        inside = ((x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N)
                  & (z + dz >= 0) & (z + dz < N))
        kf = np.where(inside, 2.0 * kap * kap[np.where(inside, nb, idx)]
                      / (kap + kap[np.where(inside, nb, idx)]), kap)
        diag += kf
        cols[:, c] = nb
        valid[:, c] = inside
        vals[:, c] = -kf
    vals[:, 3] = diag
    return _assemble(cols, vals, valid)


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """U[lo, hi) float64 samples from a seeded PCG64 stream."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def random_triangular(n: int, lower: bool, seed: int, unit: bool = False,
                      max_row: int = 48, empty_frac: float = 0.1,
                      long_frac: float = 0.05, long_row: int = 400,
                      band: int | None = None) -> CSR:
    """Random sparse triangular matrix with a mixed row-length distribution.

    Each row gets k strict entries: 0 with probability ``empty_frac``, up to
    ``long_row`` with probability ``long_frac``, otherwise U{1..max_row}; k is
    capped by the number of columns available on the strict side (within
    ``band`` of the diagonal if given).  Off-diagonals are U[-1,1]; the diagonal
    is 1 if ``unit`` else positive and dominant (1.2 .. 2 times the row's
    absolute off-diagonal sum plus 1), so that |I - D^-1 T| has row sums < 1.
    """
    rng = np.random.default_rng(seed)
    rows_c, rows_v = [], []
    for i in range(n):
        avail = i if lower else n - 1 - i
        if band is not None:
            avail = min(avail, band)
        u = rng.random()
        if u < empty_frac:
            k = 0
        elif u < empty_frac + long_frac:
            k = int(rng.integers(1, long_row + 1))
        else:
            k = int(rng.integers(1, max_row + 1))
        k = min(k, avail)
        if k > 0:
            if lower:
                lo = i - avail
                c = np.sort(rng.choice(avail, size=k, replace=False) + lo)
            else:
                c = np.sort(rng.choice(avail, size=k, replace=False) + i + 1)
        else:
            c = np.zeros(0, dtype=np.int64)
        v = rng.uniform(-1.0, 1.0, size=k)
        if unit:
            d = 1.0
            v = v / max(1.0, 1.25 * np.abs(v).sum())
        else:
            d = (np.abs(v).sum() + 1.0) * rng.uniform(1.2, 2.0)
        if lower:
            rows_c.append(np.concatenate([c, [i]]))
            rows_v.append(np.concatenate([v, [d]]))
        else:
            rows_c.append(np.concatenate([[i], c]))
            rows_v.append(np.concatenate([[d], v]))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(c) for c in rows_c])
    ci = np.concatenate(rows_c).astype(np.int32) if n else np.zeros(0, np.int32)
    va = np.concatenate(rows_v).astype(np.float64) if n else np.zeros(0)
    return CSR(n, rp.astype(np.int32), ci, va)
