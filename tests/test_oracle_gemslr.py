"""Pins for the oracle's GeMSLR setup and solve against what the paper fixes.

T1 block-LDU identity (Sec. 2.1), T2 S = C - E B^-1 F = (I - G) C (eq. gemslr1),
T3 Sherman-Morrison-Woodbury form of S^-1 (eq. gemslr4), T4 eigenvalues
gamma/(1-gamma) of the correction (Sec. 2.2), T5 full-rank exactness, T6 the
k = 0 special case, T7 linearity, T8 Arnoldi (Krylov-Schur) relation and Ritz
values, T13 basis invariance.  All on dense brute force with n <= 500.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import gemslr_inputs as gi
from oracle import OracleGemslr, multilevel_partition
from oracle.lowrank import block_eigs, correction_matrix, correction_score, krylov_schur


def _problem(dims=(7, 6, 5), beta=0.6, sigma=0.0, nlev=3, p=4, p_last=None):
    A, xyz = gi.grid_operator(dims, beta=beta, sigma=sigma)
    As = A.to_scipy()
    P = multilevel_partition(As, xyz, nlev, p, p_last)
    return As, P


def _LU(L, U):
    n = L.shape[0]
    return (np.eye(n) + L.toarray()) @ U.toarray()


def test_block_ldu_identity_T1_T2():
    As, P = _problem()
    M = OracleGemslr(As, P, ilu="ilu0", rank=0, lowrank=False)
    Ah = M.Ahat.toarray()
    lv = M.levels[0]
    s, e = lv["s"], lv["e"]
    B, F, E, C = Ah[s:e, s:e], lv["F"].toarray(), lv["E"].toarray(), Ah[e:, e:]
    assert np.array_equal(F, Ah[s:e, e:]) and np.array_equal(E, Ah[e:, s:e])
    Binv = np.linalg.inv(B)
    S = C - E @ Binv @ F
    d, sz = e - s, Ah.shape[0] - e
    I1, I2 = np.eye(d), np.eye(sz)
    Lb = np.block([[I1, np.zeros((d, sz))], [E @ Binv, I2]])
    Db = np.block([[B, np.zeros((d, sz))], [np.zeros((sz, d)), S]])
    Ub = np.block([[I1, Binv @ F], [np.zeros((sz, d)), I2]])
    assert np.allclose(Lb @ Db @ Ub, Ah, rtol=1e-12, atol=1e-9 * abs(Ah).max())
    G = E @ Binv @ F @ np.linalg.inv(C)
    assert np.allclose((I2 - G) @ C, S, atol=1e-9 * abs(S).max())


def test_smw_and_correction_eigenvalues_T3_T4():
    As, P = _problem(beta=0.3)
    M = OracleGemslr(As, P, ilu="ilu0", rank=0, lowrank=False)
    Ah = M.Ahat.toarray()
    e = M.levels[0]["e"]
    s = M.levels[0]["s"]
    B, F, E, C = Ah[s:e, s:e], Ah[s:e, e:], Ah[e:, s:e], Ah[e:, e:]
    Cinv = np.linalg.inv(C)
    G = E @ np.linalg.solve(B, F) @ Cinv
    S = C - E @ np.linalg.solve(B, F)
    R, W = sla.schur(G, output="real")
    Hc = correction_matrix(R)                      # (I - R)^-1 - I
    Sinv = Cinv + Cinv @ W @ Hc @ W.T
    assert np.allclose(Sinv, np.linalg.inv(S), rtol=1e-9, atol=1e-12 * abs(Sinv).max())
    gam = np.linalg.eigvals(G)
    corr = np.linalg.eigvals(W @ Hc @ W.T)
    expect = gam / (1 - gam)
    assert np.allclose(np.sort_complex(corr), np.sort_complex(expect), rtol=1e-8, atol=1e-10)


def _dense_full_rank(M, l):
    """A_tilde_l = [L_l U_l, F_l; E_l, A_tilde_{l+1}]; the last level is its block LU."""
    if l == M.nlev - 1:
        return _LU(M.last_L, M.last_U)
    lv = M.levels[l]
    C = _dense_full_rank(M, l + 1)
    return np.block([[_LU(lv["L"], lv["U"]), lv["F"].toarray()], [lv["E"].toarray(), C]])


def _dense_rank0(M, l):
    """k = 0: A_tilde_l = [LU, F; E, A_tilde_{l+1} + E (LU)^-1 F]."""
    if l == M.nlev - 1:
        return _LU(M.last_L, M.last_U)
    lv = M.levels[l]
    LU = _LU(lv["L"], lv["U"])
    F, E = lv["F"].toarray(), lv["E"].toarray()
    C = _dense_rank0(M, l + 1) + E @ np.linalg.solve(LU, F)
    return np.block([[LU, F], [E, C]])


def _dense_Minv(M):
    n = M.n
    I = np.eye(n)
    return np.column_stack([M.apply_perm(I[:, i]) for i in range(n)])


def _full_ranks(P):
    lp = P["level_ptr"]
    n = lp[-1]
    return [int(n - lp[l + 1]) for l in range(len(lp) - 2)]


@pytest.mark.parametrize("ilu", ["ilu0", "ilut"])
def test_full_rank_is_exact_inverse_of_A_tilde_T5(ilu):
    As, P = _problem()
    M = OracleGemslr(As, P, ilu=ilu, tau=1e-2, lfil=3, rank=_full_ranks(P))
    Minv = _dense_Minv(M)
    At = _dense_full_rank(M, 0)
    assert np.allclose(Minv @ At, np.eye(M.n), atol=1e-9)


def test_full_rank_exact_factors_gives_A_inverse_T5():
    As, P = _problem(p_last=1)
    M = OracleGemslr(As, P, ilu="exact", rank=_full_ranks(P))
    b = gi.rhs_uniform(M.n, 9)
    x = np.linalg.solve(As.toarray(), b)
    assert np.allclose(M.apply(b), x, rtol=1e-9, atol=1e-12 * abs(x).max())


def test_rank_zero_is_block_ilu_schur_solve_T6():
    As, P = _problem(beta=0.9)
    M = OracleGemslr(As, P, ilu="ilut", tau=1e-2, lfil=2, rank=0)
    Minv = _dense_Minv(M)
    assert np.allclose(Minv @ _dense_rank0(M, 0), np.eye(M.n), atol=1e-9)


def test_linearity_and_permutation_T7():
    As, P = _problem(sigma=0.02)
    M = OracleGemslr(As, P, ilu="ilu0", rank=4)
    n = M.n
    x, y = gi.rhs_uniform(n, 1), gi.rhs_uniform(n, 2)
    a, b = 0.7, -1.3
    assert np.allclose(M.apply(a * x + b * y), a * M.apply(x) + b * M.apply(y), rtol=1e-11, atol=1e-14)
    # original-order apply = P * M_hat^-1 * P^T
    Pm = np.eye(n)[:, M.perm]
    assert np.allclose(M.apply(x), Pm @ M.apply_perm(Pm.T @ x), rtol=1e-13)


def test_arnoldi_relation_and_ritz_values_T8():
    As, P = _problem(dims=(8, 8, 7), beta=0.2, nlev=2, p=4)
    M = OracleGemslr(As, P, ilu="ilu0", rank=4, lowrank=False)
    lv = M.levels[0]
    s = M.n - lv["e"]
    op = lambda z: M.g_hat(0, z)
    W, Tk, info = krylov_schur(op, s, 4, 1000, tol=1e-2)
    k = W.shape[1]
    assert s > 2 * 4 and not info["dense"]
    assert np.allclose(W.T @ W, np.eye(k), atol=1e-12)
    # restarted Arnoldi relation: G W - W T = beta v e^T Q_k, columns below the 2-digit bound
    Gd = np.column_stack([op(np.eye(s)[:, i]) for i in range(s)])
    R = Gd @ W - W @ Tk
    theta = block_eigs(Tk)
    assert np.linalg.norm(R, 2) <= 1.01e-2 * np.min(np.abs(theta)) + 1e-12
    # Ritz values agree with the wanted eigenvalues of the dense G_hat to two digits
    ev = np.linalg.eigvals(Gd)
    order = np.lexsort((-np.abs(ev), -correction_score(ev)))
    want = ev[order[:k]]
    for t in theta:
        assert np.min(np.abs(want - t)) <= 1e-2 * abs(t)


def test_basis_invariance_T13():
    As, P = _problem()
    M = OracleGemslr(As, P, ilu="ilu0", rank=3)
    x = gi.rhs_uniform(M.n, 4)
    y0 = M.apply(x)
    rng = np.random.default_rng(1)
    for lv in M.levels:
        k = lv["W"].shape[1]
        Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
        lv["W"] = lv["W"] @ Q
        lv["H"] = Q.T @ lv["H"] @ Q
    assert np.allclose(M.apply(x), y0, rtol=1e-11, atol=1e-14)


def test_wanted_selection_never_splits_a_pair():
    # rotation block: eigenvalues 0.5 +- 0.4i tie in score -> k=1 keeps both
    from oracle.lowrank import schur_wanted
    Hm = np.array([[0.5, 0.4, 0.0], [-0.4, 0.5, 0.0], [0.3, 0.2, 0.1]])
    T, Q, keff = schur_wanted(Hm, 1)
    assert keff == 2
    assert np.allclose(Q @ T @ Q.T, Hm)
    assert np.allclose(np.sort_complex(block_eigs(T[:2, :2])),
                       np.sort_complex(np.array([0.5 - 0.4j, 0.5 + 0.4j])))
    # a real value with larger |theta/(1-theta)| wins over the pair
    Hm2 = np.diag([0.9, 0.1, 0.2])
    T, Q, keff = schur_wanted(Hm2, 1)
    assert keff == 1 and np.isclose(T[0, 0], 0.9)


def test_randomized_schur_recovers_an_exact_low_rank_operator():
    """An operator of rank r <= b: the random block's range is its range, so the
    Rayleigh quotient holds its nonzero eigenvalues exactly and W spans an
    invariant subspace (G W = W T_k to rounding)."""
    from oracle.lowrank import randomized_schur
    rng = np.random.default_rng(11)
    s, r = 300, 6
    X = np.linalg.qr(rng.standard_normal((s, r)))[0]
    Yb = rng.standard_normal((s, r))
    D = np.diag([0.9, 0.8, -0.7, 0.6, 0.5, 0.4])
    G = X @ D @ (Yb.T @ X) @ np.linalg.inv(Yb.T @ X) @ X.T       # rank r, eigenvalues diag(D) and 0
    W, Tk, info = randomized_schur(lambda z: G @ z, s, r, 5, oversample=4, power=0)
    assert W.shape == (s, r) and np.allclose(W.T @ W, np.eye(r), atol=1e-12)
    assert np.linalg.norm(G @ W - W @ Tk) <= 1e-10
    ev = np.sort(np.linalg.eigvals(Tk).real)
    assert np.allclose(ev, np.sort(np.diag(D)), atol=1e-10)
    assert info["products"] == 2 * (r + 4)


def test_randomized_schur_agrees_with_arnoldi_on_the_dominant_values():
    """On G_hat of a hierarchy the subspace iteration finds the same leading
    Ritz values as the thick-restart Arnoldi to the Arnoldi's own accuracy
    (two digits), and the correction is exact at full rank like the Arnoldi's."""
    from oracle.lowrank import krylov_schur, randomized_schur
    A, xyz = gi.grid_operator((10, 9, 8), beta=0.2)
    As = A.to_scipy()
    part = multilevel_partition(As, xyz, 3, 4)
    M = OracleGemslr(As, part, ilu="ilut", tau=1e-2, lfil=4, rank=5, lowrank=False)
    lv = M.levels[0]
    s = M.n - lv["e"]
    op = lambda z: M.g_hat(0, z)           # noqa: E731
    _, _, ia = krylov_schur(op, s, 5, 1000, tol=1e-6, max_cycles=50)
    _, _, ir = randomized_schur(op, s, 5, 1000, oversample=10, power=3)
    ta = np.sort_complex(ia["ritz"])
    tr = np.sort_complex(ir["ritz"])
    assert len(ta) == len(tr)
    assert np.allclose(tr, ta, rtol=1e-2, atol=1e-3)
    # full rank: the randomized set-up reproduces the exact inverse of A~ (T5)
    A2, xyz2 = gi.grid_operator((8, 7), beta=0.3)
    A2s = A2.to_scipy()
    part2 = multilevel_partition(A2s, xyz2, 2, 2, p_last=1)
    Mr = OracleGemslr(A2s, part2, ilu="exact", rank=10 ** 6, lowrank="randomized")
    r = gi.rhs_uniform(A2.n, 3)
    assert np.allclose(Mr.apply(r), np.linalg.solve(A2s.toarray(), r), rtol=1e-8)


@pytest.mark.parametrize("shift", [0.0, 0.05])
def test_hierarchy_from_given_factors_is_the_same_operator(shift):
    """OracleGemslr.from_factors rebuilds Alg. 2 from given factors only: fed
    the factors of an oracle set-up it applies the same M^-1, bit for bit, in
    real and in complex arithmetic; fed altered factors it follows them."""
    As, P = _problem()
    M = OracleGemslr(As, P, ilu="ilut", tau=1e-2, lfil=4, rank=3, shift=shift)
    fac = M.factors()
    M2 = OracleGemslr.from_factors(As, P, fac)
    for seed in (1, 2):
        r = gi.rhs_uniform(As.shape[0], seed)
        assert np.array_equal(M2.apply(r), M.apply(r))
    fac["levels"][0]["H"] = 2.0 * fac["levels"][0]["H"]      # a different correction is followed
    M3 = OracleGemslr.from_factors(As, P, fac)
    r = gi.rhs_uniform(As.shape[0], 3)
    assert not np.allclose(M3.apply(r), M.apply(r))
