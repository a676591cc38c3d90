"""The delayed reorthogonalisation the GPU's FGMRES uses for a linear M^{-1},
restated step by step in numpy and checked against the oracle's modified
Gram-Schmidt FGMRES: after k steps of one cycle both give the same iterate.

Step j, in the order the GPU runs it:
  beside M^{-1}:  v_{j-1} = (vt_{j-1} - V_{j-2} a_{j-1}) / nu_{j-1};
                  a = V_{j-1}^T vt_j, gam = vt_j . vt_j
  after it:       z = M^{-1} vt_j (kept as column j of Zt), w = A z;
                  b = V_{j-1}^T w, dlt = vt_j . w, om = w . w
  finisher:       nu = sqrt(gam - a.a), coef = [b; (dlt - a.b) / nu],
                  btil = sqrt(om - coef.coef) / nu,
                  column j-1 of H = [h1_{j-1} + btil_{j-1} a; btil_{j-1} nu],
                  column j of R = [a; nu], h1_j = (coef - H_{j} a) / nu
  next direction: vt_{j+1} = (w - V_{j-1} (coef[:j] - a coef[j] / nu)
                              - vt_j coef[j] / nu) / (nu btil)
Cycle end: the last direction's a and nu close column k-1; y solves the least
squares problem; x = x0 + Zt R^{-1} y.  No v_j is ever needed before the step
after the next, which is what lets the GPU run its reorthogonalisation beside
M^{-1}."""
import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import fgmres
from tests.helpers import oracle_hierarchy, problem


def dcgs2_cycle(As, b, Mapply, k):
    n = len(b)
    beta0 = np.linalg.norm(b)
    V = np.zeros((n, k + 1))
    Zt = np.zeros((n, k))
    H = np.zeros((k + 1, k))
    R = np.zeros((k, k))
    vt = b / beta0                  # the first direction is exact: a = [], nu = 1
    a_prev = nu_prev = None
    hprev = btil_prev = None
    for j in range(k):
        # beside M^{-1}: fix v_{j-1}, then a and gam for vt_j
        if j > 0:
            V[:, j - 1] = (V[:, j - 1] - V[:, :j - 1] @ a_prev) / nu_prev
        a = V[:, :j].T @ vt
        gam = vt @ vt
        # the product and its reduction
        z = Mapply(vt)
        Zt[:, j] = z
        w = As @ z
        bb = V[:, :j].T @ w
        dlt = vt @ w
        om = w @ w
        # finisher
        nu = np.sqrt(max(gam - a @ a, 0.0))
        vjw = (dlt - a @ bb) / nu
        coef = np.concatenate([bb, [vjw]])
        btil = np.sqrt(max(om - coef @ coef, 0.0)) / nu
        if j > 0:
            H[:j, j - 1] = hprev + btil_prev * a
            H[j, j - 1] = btil_prev * nu
        R[:j, j] = a
        R[j, j] = nu
        g = H[:j + 1, :j] @ a if j > 0 else np.zeros(1)
        h1 = (coef - g) / nu
        # next direction from vt_j and V_{j-1}; vt_j kept in column j
        cj = coef[j] / nu
        cf = coef[:j] - a * cj
        V[:, j] = vt
        vt = (w - V[:, :j] @ cf - V[:, j] * cj) / (nu * btil)
        a_prev, nu_prev, hprev, btil_prev = a, nu, h1, btil
    # cycle end: fix v_{k-1}, close column k-1 with the last direction
    V[:, k - 1] = (V[:, k - 1] - V[:, :k - 1] @ a_prev) / nu_prev
    a = V[:, :k].T @ vt
    nu = np.sqrt(max(vt @ vt - a @ a, 0.0))
    H[:k, k - 1] = hprev + btil_prev * a
    H[k, k - 1] = btil_prev * nu
    e1 = np.zeros(k + 1)
    e1[0] = beta0
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    return Zt @ np.linalg.solve(np.triu(R), y), np.linalg.norm(e1 - H @ y) / beta0


@pytest.mark.parametrize("name,k,prec", [("c1", 8, True), ("c1", 25, True), ("small3d", 12, True),
                                         ("shifted", 15, True), ("c1", 60, False), ("c1", 100, False)])
def test_delayed_reorthogonalisation_equals_mgs_fgmres(name, k, prec):
    """With M^{-1} = I on the 2-D Laplacian (no preconditioner) the first pass
    loses orthogonality quickly, so the lagged corrections (a, and the folded
    a coef_j / nu of the next direction) matter well above rounding."""
    A, xyz, part = problem(name)
    As = A.to_scipy()
    Mapply = oracle_hierarchy(name).apply if prec else (lambda v: v.copy())
    b = gi.rhs_uniform(A.n, 31)
    x_ref, info = fgmres(As, b, Mapply, restart=k, rtol=1e-15, maxit=k)
    x, est = dcgs2_cycle(As, b, Mapply, k)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert abs(est - info["hist"][-1]) <= 1e-6 * info["hist"][-1] + 1e-15
    # the estimate is the true residual of the iterate (a linear M^{-1})
    assert abs(np.linalg.norm(b - As @ x) / np.linalg.norm(b) - est) <= 1e-6 * est + 1e-13
