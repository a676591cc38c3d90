"""Pins for the oracle's complex arithmetic, used by the complex shift of the
incomplete factorisations (Sec. 5.2.3: each on-diagonal block is factored as
B + i alpha I, alpha = 0.05 sum_i |a_ii| / n in the paper): complex ILU,
complex Krylov-Schur, complex FGMRES and the shifted hierarchy."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import gemslr_inputs as gi
from oracle import OracleGemslr, fgmres, multilevel_partition
from oracle.ilu import ilu0, ilut, lu_solve
from oracle.lowrank import krylov_schur


def _hand_matrix():
    return np.array([[10.0, 1.0, 5.0, 0.0, 0.0],
                     [4.0, 2.0, 0.0, 3.0, 0.0],
                     [1.0, 6.0, 10.0, 0.0, 1.0],
                     [0.0, 3.0, 4.0, 20.9, 4.0],
                     [5.0, 0.0, 0.0, 0.0, 10.0]])


def test_complex_ilut_phase_invariance_of_hand_case():
    """Every magnitude of the dual-threshold rule is a modulus, so ILUT of
    e^{i phi} A keeps the pattern of ILUT(A) (the hand-worked case of
    test_oracle_ilu) with L unchanged and U multiplied by e^{i phi}."""
    A = _hand_matrix()
    L, U, _ = ilut(sp.csr_matrix(A), 0.1, 1)
    ph = np.exp(0.7j)
    Lz, Uz, nc = ilut(sp.csr_matrix(ph * A), 0.1, 1)
    assert nc == 0 and Lz.dtype == np.complex128
    assert np.array_equal(Lz.toarray() != 0, L.toarray() != 0)
    assert np.allclose(Lz.toarray(), L.toarray(), rtol=1e-14, atol=1e-15)
    assert np.allclose(Uz.toarray(), ph * U.toarray(), rtol=1e-14, atol=1e-14)


def test_complex_ilu_exact_and_pattern():
    A, _ = gi.grid_operator((5, 4, 3), beta=0.3, sigma=0.1)
    B = sp.csr_matrix(A.to_scipy(), dtype=complex) + 0.4j * sp.eye(A.n, format="csr")
    D = B.toarray()
    L, U, nc = ilut(B, 0.0, -1)                       # tau = 0, no fill limit: exact LU
    assert nc == 0
    assert np.allclose((np.eye(A.n) + L.toarray()) @ U.toarray(), D, rtol=1e-12, atol=1e-10)
    b = gi.rhs_uniform(A.n, 3)
    assert np.allclose(lu_solve(L, U, b), np.linalg.solve(D, b), rtol=1e-10, atol=1e-12)
    L0, U0, _ = ilu0(B)                               # (LU)_ij = b_ij on the pattern (Saad, Prop. 10.4)
    LU = (np.eye(A.n) + L0.toarray()) @ U0.toarray()
    mask = D != 0
    assert np.allclose(LU[mask], D[mask], rtol=1e-13, atol=1e-10)


def test_complex_fgmres_is_the_krylov_minimiser():
    """After k steps with a fixed complex M, x_k minimises ||b - A x|| over
    x in M K_k(A M, b): brute force over a monomial basis."""
    rng = np.random.default_rng(4)
    n = 40
    A = sp.csr_matrix(np.diag(np.linspace(1.0, 3.0, n)) + 0.3 * rng.standard_normal((n, n)))
    Mi = np.linalg.inv(np.diag(np.linspace(1.0, 3.0, n)) + 0.5j * np.eye(n))
    b = rng.standard_normal(n)
    for k in (1, 3, 6):
        x, info = fgmres(A, b, lambda v: Mi @ v, restart=50, rtol=1e-30, maxit=k, cplx=True)
        K = [b.astype(complex)]
        for _ in range(k - 1):
            K.append(A @ (Mi @ K[-1]))
        Kb = Mi @ np.column_stack(K)
        c = np.linalg.lstsq(A @ Kb, b, rcond=None)[0]
        xb = Kb @ c
        assert np.linalg.norm(x - xb) <= 1e-8 * np.linalg.norm(xb)
        assert abs(info["hist"][-1] - np.linalg.norm(b - A @ xb) / np.linalg.norm(b)) <= 1e-8


def test_complex_fgmres_on_real_data_equals_real_fgmres():
    A, _ = gi.grid_operator((7, 6, 5), beta=0.4)
    As = A.to_scipy()
    b = gi.rhs_uniform(A.n, 5)
    d = As.diagonal()
    x1, i1 = fgmres(As, b, lambda v: v / d, restart=15, rtol=1e-10)
    x2, i2 = fgmres(As, b, lambda v: v / d, restart=15, rtol=1e-10, cplx=True)
    assert i1["iters"] == i2["iters"] and np.allclose(i1["hist"], i2["hist"], rtol=1e-10)
    assert np.allclose(x2.imag, 0.0) and np.allclose(x1, x2.real, rtol=1e-10)


def test_complex_krylov_schur_relation_and_ritz_values():
    rng = np.random.default_rng(7)
    s = 120
    # six well separated wanted values (largest |theta/(1-theta)|), the rest in a small disc
    top = np.array([0.95, 0.9, 0.85, 0.8, 0.75, 0.7]) * np.exp(1j * np.linspace(0.2, 1.2, 6))
    rest = 0.3 * np.sqrt(rng.uniform(size=s - 6)) * np.exp(2j * np.pi * rng.uniform(size=s - 6))
    S = np.eye(s) + 0.1 * (rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))) / np.sqrt(s)
    G = S @ np.diag(np.concatenate([top, rest])) @ np.linalg.inv(S)
    W, T, info = krylov_schur(lambda z: G @ z, s, 6, 1000, tol=1e-8, max_cycles=60, complex_arith=True)
    assert W.shape == (s, 6) and info["converged"]
    assert np.allclose(W.conj().T @ W, np.eye(6), atol=1e-12)
    assert np.allclose(np.tril(T, -1), 0.0)
    # W spans an invariant subspace: G W = W T up to the stopping tolerance
    assert np.linalg.norm(G @ W - W @ T) <= 1e-6 * np.linalg.norm(T)
    ev = np.linalg.eigvals(G)
    score = np.abs(ev / (1.0 - ev))
    want = ev[np.argsort(-score)[:6]]
    for t in np.diag(T):
        assert np.min(np.abs(want - t)) <= 1e-8 * max(1.0, abs(t))


def test_shifted_hierarchy_full_rank_exact_factors_is_the_shifted_inverse():
    """Every diagonal block of every level (and the single last-level block)
    is factored exactly as B + i alpha I and every correction has full rank,
    so level by level the application is the exact block elimination of
    A + i alpha I: M^{-1} = (A + i alpha I)^{-1} (the complex analogue of T5)."""
    A, xyz = gi.grid_operator((7, 6), beta=0.2, sigma=0.3)
    As = A.to_scipy()
    part = multilevel_partition(As, xyz, 3, 2, p_last=1)
    M = OracleGemslr(As, part, ilu="exact", rank=10 ** 6, shift=0.05)
    alpha = 0.05 * np.abs(As.diagonal()).sum() / A.n
    assert abs(M.alpha - alpha) <= 1e-15 * alpha
    r = gi.rhs_uniform(A.n, 6)
    z = M.apply(r)
    ref = np.linalg.solve(As.toarray() + 1j * alpha * np.eye(A.n), r)
    assert np.allclose(z, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    # shift 0 gives back the real method
    M0 = OracleGemslr(As, part, ilu="exact", rank=10 ** 6)
    assert np.allclose(M0.apply(r), np.linalg.solve(As.toarray(), r), rtol=1e-9)
