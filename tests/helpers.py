"""Shared builders for the tests (oracle hierarchies on seeded problems)."""
import functools

import numpy as np

import gemslr_inputs as gi
from oracle import OracleGemslr, local_order, multilevel_partition

CASES = {
    # name: (dims, beta, sigma, nlev, p, ilu, tau, lfil, rank)
    "c1": ((32, 32), 0.0, 0.0, 2, 4, "ilu0", 0.0, 0, 8),
    "small3d": ((13, 11, 9), 0.4, 0.0, 3, 8, "ilut", 1e-2, 5, 5),
    "shifted": ((12, 12, 12), 0.0, 0.05, 4, 8, "ilut", 1e-3, 10, 6),
    "rank0": ((10, 9, 8), 0.2, 0.0, 3, 4, "ilu0", 0.0, 0, 0),
    "tinyparts": ((6, 5, 4), 0.3, 0.0, 3, 16, "ilu0", 0.0, 0, 3),
    "bigblock": ((240, 240), 0.5, 0.0, 2, 2, "ilu0", 0.0, 0, 4),
    "c2": ((64, 64, 64), 0.1, 0.0, 4, 64, "ilut", 1e-3, 10, 32),
    # the benchmarked 64^3 workload: interface levels in the local multicolour order
    "c2local": ((64, 64, 64), 0.1, 0.0, 4, 64, "ilut", 1e-3, 10, 32),
    # indefinite (shift 0.1 h^-2): the DGKS test skips the second Gram-Schmidt
    # pass at step 7 of the first cycle, every other step takes it
    "indef24": ((24, 24, 24), 0.0, 0.1, 4, 8, "ilut", 1e-3, 10, 8),
    # the indefinite operators of the 128^3 and 96^3 workloads (shifts -0.05 h^-2
    # and -0.1 h^-2) at a size the oracle solves in seconds
    "indef32a": ((32, 32, 32), 0.0, 0.05, 4, 8, "ilut", 1e-3, 10, 32),
    "indef32b": ((32, 32, 32), 0.0, 0.1, 4, 8, "ilut", 1e-3, 10, 32),
    # a 5-unknown root Schur system: 8 inner GMRES steps end in a happy breakdown
    "tiny2d": ((9, 5), 0.3, 0.0, 2, 2, "ilu0", 0.0, 0, 2),
}


LOCAL_FROM = {"c2local": 1}


@functools.lru_cache(maxsize=None)
def problem(name):
    dims, beta, sigma, nlev, p, ilu, tau, lfil, rank = CASES[name]
    A, xyz = gi.grid_operator(dims, beta=beta, sigma=sigma)
    part = multilevel_partition(A.to_scipy(), xyz, nlev, p)
    if name in LOCAL_FROM:
        part = local_order(part, xyz, LOCAL_FROM[name])
    return A, xyz, part


@functools.lru_cache(maxsize=None)
def oracle_hierarchy(name):
    dims, beta, sigma, nlev, p, ilu, tau, lfil, rank = CASES[name]
    A, xyz, part = problem(name)
    return OracleGemslr(A.to_scipy(), part, ilu=ilu, tau=tau, lfil=lfil, rank=rank)


def lib_opts(name):
    dims, beta, sigma, nlev, p, ilu, tau, lfil, rank = CASES[name]
    return dict(ilu=ilu, tau=tau, lfil=lfil, rank=rank)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16(a):
    """Round float64 -> float32 -> bfloat16 (nearest even) -> float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_w_to_bf16(M):
    """Replace every W_l of an oracle hierarchy by its BF16-rounded copy (in place),
    so that a mixed-precision GPU application of the same factors differs from
    the FP64 oracle by FP32 rounding only; returns M.factors()."""
    for lv in M.levels:
        lv["W"] = bf16(lv["W"])
    return M.factors()


@functools.lru_cache(maxsize=None)
def oracle_hierarchy_z(name, shift):
    """Oracle hierarchy of a case with the complex diagonal shift (Sec. 5.2.3)."""
    dims, beta, sigma, nlev, p, ilu, tau, lfil, rank = CASES[name]
    A, xyz, part = problem(name)
    return OracleGemslr(A.to_scipy(), part, ilu=ilu, tau=tau, lfil=lfil, rank=rank, shift=shift)


def rhs_complex(n, seed):
    """Seeded complex right-hand side: real and imaginary parts U[-1, 1)."""
    return gi.rhs_uniform(n, seed) + 1j * gi.rhs_uniform(n, seed + 1000)
