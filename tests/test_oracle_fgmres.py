"""Pins for the oracle's FGMRES (T11, T12) and an end-to-end check on c1."""
import numpy as np
import scipy.linalg as sla

import gemslr_inputs as gi
from oracle import OracleGemslr, fgmres, multilevel_partition


def _small(n=40, seed=0):
    A, _ = gi.grid_operator((8, 5), beta=3.0)
    return A.to_scipy(), gi.rhs_uniform(A.n, seed)


def test_minimal_residual_over_krylov_space():
    # with M = I, step j of GMRES minimises ||b - A x|| over K_j(A, b) (brute force)
    A, b = _small()
    Ad = A.toarray()
    bn = np.linalg.norm(b)
    for j in (1, 3, 7, 12):
        x, info = fgmres(A, b, lambda v: v, restart=j, rtol=1e-300, maxit=j)
        K = np.column_stack([np.linalg.matrix_power(Ad, i) @ b for i in range(j)])
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(Ad @ Q, b, rcond=None)[0]
        best = np.linalg.norm(b - Ad @ (Q @ y))
        assert np.isclose(np.linalg.norm(b - A @ x), best, rtol=1e-8)
        assert np.isclose(info["hist"][-1], best / bn, rtol=1e-8)


def test_monotone_residual_and_dense_solution_T11_T12():
    A, xyz = gi.grid_operator((9, 8, 6), beta=0.5, sigma=0.01)
    As = A.to_scipy()
    b = gi.rhs_uniform(A.n, 3)
    P = multilevel_partition(As, xyz, 3, 4)
    M = OracleGemslr(As, P, ilu="ilut", tau=1e-2, lfil=4, rank=6)
    x, info = fgmres(As, b, M.apply, restart=10, rtol=1e-10)
    assert info["converged"] and info["restarts"] >= 1
    h = np.array(info["hist"])
    assert np.all(np.diff(h) <= 1e-12)       # non-increasing within and across cycles
    xd = sla.solve(As.toarray(), b)
    cond = np.linalg.cond(As.toarray())
    assert np.linalg.norm(x - xd) <= 1e-10 * cond * np.linalg.norm(xd)
    assert np.linalg.norm(b - As @ x) <= 1e-10 * np.linalg.norm(b)


def test_flexible_equals_right_preconditioned_gmres_for_fixed_M():
    A, xyz = gi.grid_operator((10, 9), beta=1.0)
    As = A.to_scipy()
    b = gi.rhs_uniform(A.n, 5)
    P = multilevel_partition(As, xyz, 2, 4)
    M = OracleGemslr(As, P, ilu="ilu0", rank=4)
    x1, i1 = fgmres(As, b, M.apply, restart=8, rtol=1e-9, flexible=True)
    x2, i2 = fgmres(As, b, M.apply, restart=8, rtol=1e-9, flexible=False)
    assert i1["iters"] == i2["iters"]
    assert np.allclose(i1["hist"], i2["hist"], rtol=1e-7)
    assert np.allclose(x1, x2, rtol=1e-7, atol=1e-12)


def test_c1_converges_and_low_rank_helps():
    A, xyz, b = gi.config_problem("c1")
    As = A.to_scipy()
    P = multilevel_partition(As, xyz, 2, 4)
    M8 = OracleGemslr(As, P, ilu="ilu0", rank=8)
    M0 = OracleGemslr(As, P, ilu="ilu0", rank=0)
    x8, i8 = fgmres(As, b, M8.apply, restart=30, rtol=1e-8)
    x0, i0 = fgmres(As, b, M0.apply, restart=30, rtol=1e-8)
    xn, inn = fgmres(As, b, lambda v: v, restart=30, rtol=1e-8)
    assert i8["converged"] and i8["rel_res_true"] <= 1e-8
    assert i8["iters"] <= i0["iters"] < inn["iters"]
