"""Pins for the oracle's inner GMRES at level 0 (Alg. 2 step 9).

At the root level the standard application y2 = M_S^-1 z2 (eq. gemslr6 followed by
the levels below) is replaced by k steps of GMRES on S_hat_0 y2 = z2, right
preconditioned by M_S^-1, where S_hat_0 = C_0 - E_0 U^-1 L^-1 F_0 is the
inexact Schur complement of Sec. 2.4.  The pins: the minimiser over the
Krylov space formed densely from a monomial basis (brute force), the exact
inverse of A when the factors are exact and k reaches the size of the Schur
system (GMRES terminates), and the monotone residual of GMRES in k.
"""
import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import OracleGemslr, fgmres, multilevel_partition


def _problem(dims, beta=0.4, sigma=0.0, nlev=3, p=4, p_last=None):
    A, xyz = gi.grid_operator(dims, beta=beta, sigma=sigma)
    As = A.to_scipy()
    return As, multilevel_partition(As, xyz, nlev, p, p_last)


def _dense_pieces(M):
    """S_hat_0 and M_S^-1 of level 0 as dense matrices, from the blocks of A_hat."""
    Ah = M.Ahat.toarray()
    lv = M.levels[0]
    s, e = lv["s"], lv["e"]
    LU = (np.eye(e - s) + lv["L"].toarray()) @ lv["U"].toarray()
    F, E, C = Ah[s:e, e:], Ah[e:, s:e], Ah[e:, e:]
    S_hat = C - E @ np.linalg.solve(LU, F)
    m = M.n - e
    I = np.eye(m)
    P = np.column_stack([M.precond_schur(I[:, i], 0) for i in range(m)])
    return Ah, LU, F, E, S_hat, P


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_inner_gmres_is_the_krylov_minimiser(k):
    """y2 = P K c with K = [z, (S P) z, ..., (S P)^{k-1} z] and c minimising
    ||z - S P K c||: the definition of k steps of right-preconditioned GMRES
    from y = 0, evaluated on a monomial basis with a dense least-squares
    solve, against the oracle's Arnoldi form; also the whole application."""
    As, P_ = _problem((7, 6, 5), beta=0.5, sigma=0.03)
    M = OracleGemslr(As, P_, ilu="ilut", tau=1e-2, lfil=3, rank=4, inner_steps=k)
    Ah, LU, F, E, S_hat, P = _dense_pieces(M)
    lv = M.levels[0]
    d = lv["e"] - lv["s"]
    b = gi.rhs_uniform(M.n, 11)
    z1 = np.linalg.solve(LU, b[:d])
    z2 = b[d:] - E @ z1
    K = [z2]
    for _ in range(k - 1):
        K.append(S_hat @ (P @ K[-1]))
    K = np.column_stack(K)
    c = np.linalg.lstsq(S_hat @ P @ K, z2, rcond=None)[0]
    y2 = P @ (K @ c)
    assert np.allclose(M.inner_gmres(z2, k), y2, rtol=1e-8, atol=1e-10 * abs(y2).max())
    y1 = z1 - np.linalg.solve(LU, F @ y2)
    expect = np.concatenate([y1, y2])
    assert np.allclose(M.apply_perm(b), expect, rtol=1e-8, atol=1e-10 * abs(expect).max())


def test_inner_gmres_with_exact_factors_reaches_A_inverse():
    """Exact factors make S_hat_0 the exact Schur complement (Sec. 2.1); GMRES
    with as many steps as the Schur system has unknowns solves it exactly,
    so the block-LU solve of Alg. 2 returns A^-1 b, whatever the levels below
    (here rank 0).  The early stop on a happy breakdown is part of the path."""
    As, P_ = _problem((6, 5, 4), beta=0.7, nlev=3, p=2)
    M0 = OracleGemslr(As, P_, ilu="exact", rank=0)
    m = M0.n - M0.levels[0]["e"]
    assert 4 <= m <= 60
    M = OracleGemslr(As, P_, ilu="exact", rank=0, inner_steps=m)
    b = gi.rhs_uniform(M.n, 12)
    x = np.linalg.solve(As.toarray(), b)
    assert np.allclose(M.apply(b), x, rtol=1e-9, atol=1e-11 * abs(x).max())
    # the standard application (no inner steps) is not exact with rank 0
    assert not np.allclose(M0.apply(b), x, rtol=1e-6, atol=1e-8 * abs(x).max())


def test_inner_gmres_residual_is_monotone():
    """GMRES minimises the residual over nested spaces: ||z2 - S_hat y2(k)||
    is non-increasing in k and below ||z2||."""
    As, P_ = _problem((8, 7, 6), beta=0.2, sigma=0.08)
    M = OracleGemslr(As, P_, ilu="ilut", tau=1e-2, lfil=3, rank=6)
    z2 = gi.rhs_uniform(M.n - M.levels[0]["e"], 13)
    res = [np.linalg.norm(z2)]
    for k in range(1, 8):
        res.append(np.linalg.norm(z2 - M.s_hat(M.inner_gmres(z2, k), 0)))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))
    assert res[-1] < 0.5 * res[0]


def test_fgmres_with_inner_steps_converges_on_indefinite_operator():
    """The application with inner steps is nonlinear in r; flexible GMRES
    still converges to the true residual tolerance, in fewer outer
    iterations than the standard application on a shifted operator."""
    As, P_ = _problem((14, 13, 12), beta=0.0, sigma=0.1, nlev=3, p=8)
    b = gi.rhs_uniform(As.shape[0], 14)
    its = {}
    for k in (0, 3):
        M = OracleGemslr(As, P_, ilu="ilut", tau=1e-3, lfil=10, rank=8, inner_steps=k)
        x, info = fgmres(As, b, M.apply, restart=30, rtol=1e-8, maxit=400)
        assert info["converged"]
        assert np.linalg.norm(b - As @ x) <= 1e-8 * np.linalg.norm(b)
        its[k] = info["iters"]
    assert its[3] < its[0]


def test_cgs2_arnoldi_with_pythagorean_norm_equals_mgs():
    """The GPU runs the inner Arnoldi with classical Gram-Schmidt and a second
    pass, taking h_{j+1,j} = (||w'||^2 - ||h2||^2)^(1/2) after the second
    projection instead of a third reduction.  Restated here in numpy, it gives
    the oracle's (modified Gram-Schmidt) inner GMRES result to rounding."""
    As, P_ = _problem((8, 7, 6), beta=0.3, sigma=0.06)
    M = OracleGemslr(As, P_, ilu="ilut", tau=1e-2, lfil=3, rank=6)
    z2 = gi.rhs_uniform(M.n - M.levels[0]["e"], 15)
    for k in (1, 4, 8):
        beta = np.linalg.norm(z2)
        V = [z2 / beta]
        Z = []
        H = np.zeros((k + 1, k))
        steps = k
        for j in range(k):
            Z.append(M.precond_schur(V[j], 0))
            w = M.s_hat(Z[j], 0)
            w0 = np.linalg.norm(w)
            Vj = np.column_stack(V)
            h = Vj.T @ w
            w = w - Vj @ h
            h2 = Vj.T @ w
            hn = np.sqrt(max(w @ w - h2 @ h2, 0.0))
            H[:j + 1, j] = h + h2
            H[j + 1, j] = hn
            if not hn > 1e-14 * w0:
                steps = j + 1
                break
            V.append((w - Vj @ h2) / hn)
        rhs = np.zeros(steps + 1)
        rhs[0] = beta
        c = np.linalg.lstsq(H[:steps + 1, :steps], rhs, rcond=None)[0]
        y2 = np.column_stack(Z[:steps]) @ c
        ref = M.inner_gmres(z2, k)
        assert np.allclose(y2, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max()), k
