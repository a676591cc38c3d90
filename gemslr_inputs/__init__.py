"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module defines the *problems*, not the method: the finite-difference
operators of the model problem -Lap(u) + beta*(1,1,1).grad(u) - c*u = f on the
unit square/cube (the paper's Sec. 5.1 model problem, 7-point stencil), the
grid coordinates of every unknown, and the uniform[-1,1) right-hand sides.
It holds none of the preconditioner's arithmetic (no partitioning, no
factorisation, no Krylov step) and imports nothing from ``oracle`` or from
the CUDA package, so both sides may use it.

Conventions (shared by every config):
  * unknown (i, j, k) of an nx x ny x nz grid has index i + nx*j + nx*ny*k;
  * spacing h_a = 1/(n_a + 1) per axis, homogeneous Dirichlet boundary;
  * row = sum_a h_a^-2 * (2 u_c - u_{-a} - u_{+a})
          + beta/(2 h_a) * (u_{+a} - u_{-a})  - sigma * h^-2 * u_c
    where the shift uses the spacing of the first axis (the grids it is
    used on are cubic);
  * CSR: int64 row pointer, int32 column indices sorted ascending, float64 values.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014): state += golden
gamma, then the variant-13 finaliser; u = (z >> 11) * 2^-53 in [0, 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR", "grid_operator", "laplace2d", "stencil3d", "splitmix64",
    "uniform01", "rhs_uniform", "batch_systems", "CONFIGS", "config_problem",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class CSR:
    """Plain CSR container (host, 0-based)."""

    def __init__(self, n, rowptr, colind, val):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))

    def to_dense(self):
        return self.to_scipy().toarray()


def splitmix64(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of splitmix64 seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): (splitmix64 >> 11) * 2^-53."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rhs_uniform(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand side b = 2u - 1 ~ uniform[-1, 1); shape (n,) or (nrhs, n)."""
    b = 2.0 * uniform01(seed, n * nrhs) - 1.0
    return b if nrhs == 1 else b.reshape(nrhs, n)


def grid_operator(dims, beta=0.0, sigma=0.0):
    """Finite-difference operator on a 2-D/3-D grid; returns (CSR, coords).

    ``coords`` is an (n, 3) int32 array of grid coordinates (z = 0 in 2-D).
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    h = [1.0 / (d + 1) for d in dims]
    idx = np.arange(n, dtype=np.int64)
    coords = np.zeros((n, 3), dtype=np.int32)
    stride = 1
    strides = []
    for a, d in enumerate(dims):
        coords[:, a] = (idx // stride) % d
        strides.append(stride)
        stride *= d
    diag = np.full(n, sum(2.0 / (ha * ha) for ha in h)) - sigma / (h[0] * h[0])
    rows = [idx]
    cols = [idx]
    vals = [diag]
    for a in range(nd):
        ha = h[a]
        for sgn in (-1, +1):
            c = coords[:, a].astype(np.int64) + sgn
            ok = (c >= 0) & (c < dims[a])
            r = idx[ok]
            rows.append(r)
            cols.append(r + sgn * strides[a])
            vals.append(np.full(r.size, -1.0 / (ha * ha) + sgn * beta / (2.0 * ha)))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr, cols.astype(np.int32), vals), coords


def laplace2d(N):
    """5-point Laplacian on an N x N grid."""
    return grid_operator((N, N))


def stencil3d(N, beta=0.0, sigma=0.0, dims=None):
    """7-point operator on N^3 (or ``dims``) with convection beta and shift sigma*h^-2."""
    return grid_operator(dims if dims is not None else (N, N, N), beta=beta, sigma=sigma)


def batch_systems(count=96, seed=3, lo=16, hi=48):
    """Grid sides and convection for the batched workload.

    Draw 4*count uniforms u from splitmix64(seed): system s takes
    (nx, ny, nz) = lo + floor(u * (hi - lo + 1)) from u[4s:4s+3] and
    beta = 0.5 * u[4s+3].
    """
    u = uniform01(seed, 4 * count).reshape(count, 4)
    sides = lo + np.floor(u[:, :3] * (hi - lo + 1)).astype(np.int64)
    beta = 0.5 * u[:, 3]
    return [(tuple(int(v) for v in sides[s]), float(beta[s])) for s in range(count)]


# The five workloads: operator, partition shape, factor kind, rank, solver.
# nlev counts the Schur levels plus the last (block-Jacobi) level; local_from:
# the first level whose blocks take the local multicolour order (None: none).
CONFIGS = {
    "c1": dict(kind="2d", N=32, beta=0.0, sigma=0.0, nlev=2, p=4, ilu="ilu0",
               tau=0.0, lfil=0, rank=8, restart=30, rtol=1e-8, seed=0),
    "c2": dict(kind="3d", N=64, beta=0.1, sigma=0.0, nlev=4, p=64, ilu="ilut",
               tau=1e-3, lfil=10, rank=32, restart=50, rtol=1e-8, seed=1, local_from=1),
    "c3": dict(kind="3d", N=128, beta=0.0, sigma=0.05, nlev=4, p=64, ilu="ilut",
               tau=1e-3, lfil=10, rank=64, restart=60, rtol=1e-8, seed=2, local_from=1),
    "c4": dict(kind="batch", count=96, nlev=3, p=8, ilu="ilut", tau=1e-3, lfil=10,
               rank=16, restart=50, rtol=1e-8, seed=3, nrhs=8),
    "c5": dict(kind="3d", N=96, beta=0.0, sigma=0.1, nlev=4, p=64, ilu="ilut",
               tau=1e-3, lfil=10, rank=32, restart=60, rtol=1e-8, seed=4, local_from=1),
}


def config_problem(name):
    """(CSR, coords, b) for a single-system config."""
    c = CONFIGS[name]
    if c["kind"] == "2d":
        A, xyz = laplace2d(c["N"])
    else:
        A, xyz = stencil3d(c["N"], beta=c["beta"], sigma=c["sigma"])
    return A, xyz, rhs_uniform(A.n, c["seed"])
