"""Pins for the oracle's incomplete factorisations (T10) and substitutions."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import gemslr_inputs as gi
from oracle.ilu import ilu0, ilut, lu_solve


def _block(n=7, beta=0.4, sigma=0.0):
    A, _ = gi.grid_operator((n, n - 1, 3), beta=beta, sigma=sigma)
    return A.to_scipy()


def test_ilu0_pattern_identity():
    # (LU)_ij = a_ij for every (i, j) in the pattern of A (Saad 2003, Prop. 10.4)
    B = _block()
    L, U, nc = ilu0(B)
    assert nc == 0
    n = B.shape[0]
    LU = ((sp.eye(n) + L) @ U).toarray()
    D = B.toarray()
    mask = D != 0
    assert np.allclose(LU[mask], D[mask], rtol=1e-13, atol=1e-10 * abs(D).max())
    # factors stay on the pattern: strictly lower / upper parts of A
    assert set(zip(*L.nonzero())) <= set(zip(*np.nonzero(np.tril(D, -1))))
    assert set(zip(*U.nonzero())) <= set(zip(*np.nonzero(np.triu(D))))


def test_ilut_no_dropping_is_exact_lu():
    # ILUT with tau = 0 and no fill limit is Gaussian elimination without pivoting
    B = _block(6, beta=0.9)
    L, U, nc = ilut(B, 0.0, -1)
    n = B.shape[0]
    Ld = np.eye(n) + L.toarray()
    Ud = U.toarray()
    assert np.allclose(np.tril(Ld, -1), Ld - np.eye(n))
    assert np.allclose(np.triu(Ud), Ud)
    assert np.allclose(Ld @ Ud, B.toarray(), rtol=1e-12, atol=1e-9 * abs(B).max())
    # and its solve is the exact solve
    b = gi.rhs_uniform(n, 11)
    assert np.allclose(lu_solve(L, U, b), sla.solve(B.toarray(), b), rtol=1e-10)


def test_ilut_drop_and_fill_rules():
    B = _block(8, beta=0.2)
    n = B.shape[0]
    L, U, _ = ilut(B, 1e-3, 4)
    Lr = np.diff(L.indptr)
    Ur = np.diff(U.indptr)
    assert Lr.max() <= 4 and Ur.max() <= 5          # lfil + the diagonal in U
    assert np.all(U.diagonal() != 0)
    # a huge threshold drops every off-diagonal multiplier: L = 0, U = diag(B)
    L2, U2, _ = ilut(B, 1e6, 10)
    assert L2.nnz == 0
    assert np.allclose(U2.toarray(), np.diag(B.diagonal()))
    # scale invariance of the rule: ILUT(c*B) = (L, c*U)
    L3, U3, _ = ilut(B * 1e5, 1e-3, 4)
    assert np.array_equal(L3.indices, L.indices) and np.allclose(L3.data, L.data)
    assert np.allclose(U3.data, 1e5 * U.data)
    # more fill never hurts accuracy on this block
    b = gi.rhs_uniform(n, 3)
    x = sla.solve(B.toarray(), b)
    errs = []
    for lfil in (1, 3, 10, -1):
        La, Ua, _ = ilut(B, 1e-6, lfil)
        errs.append(np.linalg.norm(lu_solve(La, Ua, b) - x))
    assert errs[-1] < 1e-5 * np.linalg.norm(x)
    assert errs[0] >= errs[-1]


def test_pivot_clamp_counts():
    # zero pivot in row 1 after elimination: [[1,1],[1,1]]
    B = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, 1.0]]))
    L, U, nc = ilu0(B)
    assert nc == 1
    assert np.isclose(U[1, 1], 1e-12 * np.sqrt(2.0))
    L, U, nc = ilut(B, 0.0, -1)
    assert nc == 1


def test_triangular_solves_match_dense():
    B = _block(5, beta=0.5, sigma=0.02)
    L, U, _ = ilut(B, 1e-2, 3)
    n = B.shape[0]
    b = gi.rhs_uniform(n, 5)
    Ld = np.eye(n) + L.toarray()
    ref = sla.solve_triangular(U.toarray(), sla.solve_triangular(Ld, b, lower=True, unit_diagonal=True))
    assert np.allclose(lu_solve(L, U, b), ref, rtol=1e-12)
