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


def test_ilut_hand_worked_dual_threshold():
    """ILUT(tau = 0.1, lfil = 1) of a 5 x 5 matrix, worked by hand from the
    dual-threshold definition (Saad's ILUT, cited in Sec. 2.1) with the
    scale-free measures of the oracle: a multiplier l_ik is measured by
    |l_ik u_kk| (the entry w_k it eliminates), a U entry by |u_ij|, both
    against tau ||a_i||_2.  The case exercises each rule so that a plausible
    misreading changes the factors:
      - final-row drop in U: row 0 drops u_01 = 1 < 1.122; kept, it would
        make u_11 = 2 - 0.4 * 1 = 1.6 instead of 2;
      - lfil selection in U: row 1 has candidates u_13 = 3 and the fill
        u_12 = -2, keeps the larger;
      - in-elimination drop: row 2 drops w_0 = 1 < 1.175 before it is used;
        used, it would make u_22 = 10 - 0.1 * 5 = 9.5;
      - keep the largest by |l_ik u_kk|, not by |l_ik|: row 3 has l_31 = 1.5
        (measure 1.5 * 2 = 3) and l_32 = 0.4 (measure 0.4 * 10 = 4) and keeps
        l_32; keeping the largest |l| or the smallest measure keeps l_31;
        measuring |l_ik| in the elimination would drop both (1.5, 0.4 < 2.19)
        and leave u_33 = 20.9;
      - fill that appears is eliminated in turn: row 4 eliminates the fill at
        columns 2 and 3 created by row 0 and row 2, which reaches u_44.
    """
    A = np.array([[10.0, 1.0, 5.0, 0.0, 0.0],
                  [4.0, 2.0, 0.0, 3.0, 0.0],
                  [1.0, 6.0, 10.0, 0.0, 1.0],
                  [0.0, 3.0, 4.0, 20.9, 4.0],
                  [5.0, 0.0, 0.0, 0.0, 10.0]])
    # row 0: thr = 0.1 sqrt(126) = 1.122.  U candidates 1 (dropped), 5.
    # row 1: thr = 0.1 sqrt(29) = 0.539.  k = 0: w_0 = 4 -> l_10 = 0.4;
    #        w_2 = -0.4 * 5 = -2 (fill).  U candidates 3 (col 3), -2 (col 2):
    #        lfil = 1 keeps col 3.  u_11 = 2.
    # row 2: thr = 0.1 sqrt(138) = 1.175.  k = 0: w_0 = 1 < thr, dropped.
    #        k = 1: l_21 = 6 / 2 = 3; w_3 = -3 * 3 = -9.  u_22 = 10; U
    #        candidates -9 (col 3), 1 (col 4, < thr, dropped).
    # row 3: thr = 0.1 sqrt(9 + 16 + 20.9^2 + 16) = 2.186.  k = 1: l_31 = 1.5,
    #        w_3 = 20.9 - 1.5 * 3 = 16.4.  k = 2: l_32 = 0.4,
    #        w_3 = 16.4 - 0.4 * (-9) = 20.  L keeps l_32 (measure 4 > 3).
    #        u_33 = 20, u_34 = 4.
    # row 4: thr = 0.1 sqrt(125) = 1.118.  k = 0: l_40 = 0.5, w_2 = -2.5
    #        (fill).  k = 2: l_42 = -2.5 / 10 = -0.25, w_3 = -0.25 * 9 = -2.25
    #        (fill).  k = 3: l_43 = -2.25 / 20 = -0.1125,
    #        w_4 = 10 + 0.1125 * 4 = 10.45.  L measures 5, 2.5, 2.25: keeps l_40.
    L_hand = np.zeros((5, 5))
    L_hand[1, 0] = 0.4
    L_hand[2, 1] = 3.0
    L_hand[3, 2] = 0.4
    L_hand[4, 0] = 0.5
    U_hand = np.zeros((5, 5))
    U_hand[0, 0], U_hand[0, 2] = 10.0, 5.0
    U_hand[1, 1], U_hand[1, 3] = 2.0, 3.0
    U_hand[2, 2], U_hand[2, 3] = 10.0, -9.0
    U_hand[3, 3], U_hand[3, 4] = 20.0, 4.0
    U_hand[4, 4] = 10.45
    L, U, nc = ilut(sp.csr_matrix(A), 0.1, 1)
    assert nc == 0
    Ld, Ud = L.toarray(), U.toarray()
    assert np.array_equal(Ld != 0, L_hand != 0)
    assert np.array_equal(Ud != 0, U_hand != 0)
    assert np.allclose(Ld, L_hand, rtol=1e-14, atol=0.0)
    assert np.allclose(Ud, U_hand, rtol=1e-14, atol=0.0)
    # U stores the diagonal first in each row, then ascending columns
    for i in range(5):
        cols = U.indices[U.indptr[i]:U.indptr[i + 1]]
        assert cols[0] == i and np.all(np.diff(cols) > 0)
