"""Rank-k Schur corrections W_{l,k}, H_l = (I - R_{l,k})^{-1} - I (Sec. 2.2-2.4).

Eq. (gemslr6): M^{-1} = C^{-1} + C^{-1} W_k [(I - R_k)^{-1} - I] W_k^H with W_k
the leading k Schur vectors of G = E B^{-1} F C^{-1}; Sec. 2.3: in practice G
is replaced by G_hat = E (U^{-1} L^{-1}) F C^{-1}, and W, R come from an
m-step Arnoldi relation G_hat V_m = V_m H_m + beta v_{m+1} e_m^T followed by
a Schur decomposition H_m = Q T Q^H, W_k = V_m Q_k, R_k = T_k.

Readings where the paper leaves details open (Sec. 4.2, Sec. 5 set-up):
  * "leading" Schur vectors: the Ritz values theta are ranked by
    |theta / (1 - theta)| descending -- the modulus of the correction's
    eigenvalue gamma/(1-gamma) (Sec. 2.2) -- ties by larger |theta|, then by
    position; a complex-conjugate pair is never split (k_eff = k + 1 then).
    Real Schur forms are used throughout (real data).
  * Arnoldi: start vector v_1 = 2u - 1 from splitmix64(1000 + l), normalised;
    classical Gram-Schmidt with one re-orthogonalisation; cycle length
    m = 2k; thick restart in Krylov-Schur form keeping the k_eff wanted Schur
    vectors; converged when the residual of the wanted invariant subspace,
    ||beta * Q[m-1, :k_eff]||_2, is at most 1e-2 * min_i |theta_i| (every
    wanted Ritz value to about two digits; the criterion does not depend on
    the basis chosen for the subspace); at most 20 cycles.
  * When s_l <= m the operator is formed densely (s_l applications to unit
    vectors) and its full real Schur form is used.
  * Complex arithmetic (the complex-shifted factors of Sec. 5.2.3 make G_hat
    complex): V^H w inner products and the complex Schur form H_m = Q T Q^H
    (the form Sec. 2.2 states); values are ranked by the same score and
    exactly k are kept (no conjugate pairs exist to keep whole).
"""
import numpy as np
import scipy.linalg as sla

import gemslr_inputs


def correction_score(theta):
    """|theta / (1 - theta)| (infinite at theta = 1)."""
    theta = np.asarray(theta, dtype=complex)
    den = np.abs(1.0 - theta)
    with np.errstate(divide="ignore"):
        return np.where(den == 0.0, np.inf, np.abs(theta) / np.where(den == 0.0, 1.0, den))


def block_eigs(T):
    """Eigenvalue of each diagonal position of a real quasi-triangular T."""
    m = T.shape[0]
    ev = np.zeros(m, dtype=complex)
    i = 0
    while i < m:
        if i + 1 < m and T[i + 1, i] != 0.0:
            a, b, c, d = T[i, i], T[i, i + 1], T[i + 1, i], T[i + 1, i + 1]
            tr, det = a + d, a * d - b * c
            disc = complex(tr * tr / 4.0 - det)
            r = np.sqrt(disc)
            ev[i] = tr / 2.0 + r
            ev[i + 1] = tr / 2.0 - r
            i += 2
        else:
            ev[i] = T[i, i]
            i += 1
    return ev


def select_wanted(theta, k):
    """Indices (into ``theta``) of the k wanted values, extended to keep pairs whole."""
    m = len(theta)
    k = min(k, m)
    if k <= 0:
        return np.zeros(0, dtype=np.int64)
    sc = correction_score(theta)
    order = np.lexsort((np.arange(m), -np.abs(theta), -sc))
    sel = list(order[:k])
    last = theta[sel[-1]]
    if last.imag != 0.0:
        # partner: the conjugate value not yet selected
        for j in order[k:]:
            if np.isclose(theta[j], np.conj(last), rtol=1e-10, atol=0.0):
                sel.append(j)
                break
    return np.array(sel, dtype=np.int64)


def schur_wanted(Hm, k):
    """Real Schur form of Hm with the wanted k (or k+1) values leading.

    Returns (T, Q, keff) with Hm = Q T Q^T and T[:keff,:keff] holding exactly
    the wanted eigenvalues.
    """
    m = Hm.shape[0]
    if k >= m:
        T, Q = sla.schur(Hm, output="real")
        return T, Q, m
    T0, _ = sla.schur(Hm, output="real")
    theta = block_eigs(T0)
    sel = select_wanted(theta, k)
    keff = len(sel)
    sc = correction_score(theta)
    inside = sc[sel].min()
    rest = np.setdiff1d(np.arange(m), sel)
    outside = sc[rest].max() if len(rest) else -np.inf
    if not inside > outside:
        raise ValueError("wanted set not separable by the correction score")
    thr = 0.5 * (inside + outside) if np.isfinite(inside) else outside * 2.0 + 1.0

    def pick(re, im):
        return correction_score(complex(re, im)) > thr

    T, Q, sdim = sla.schur(Hm, output="real", sort=pick)
    if sdim != keff:
        raise ValueError(f"reordered Schur form selected {sdim} values, expected {keff}")
    return T, Q, keff


def schur_wanted_complex(Hm, k):
    """Complex Schur form Hm = Q T Q^H with the k wanted values leading."""
    m = Hm.shape[0]
    if k >= m:
        T, Q = sla.schur(Hm.astype(complex), output="complex")
        return T, Q, m
    T0, _ = sla.schur(Hm.astype(complex), output="complex")
    theta = np.diag(T0)
    sc = correction_score(theta)
    order = np.lexsort((np.arange(m), -np.abs(theta), -sc))
    sel, rest = order[:k], order[k:]
    inside, outside = sc[sel].min(), sc[rest].max()
    if not inside > outside:
        raise ValueError("wanted set not separable by the correction score")
    thr = 0.5 * (inside + outside) if np.isfinite(inside) else outside * 2.0 + 1.0
    T, Q, sdim = sla.schur(Hm.astype(complex), output="complex", sort=lambda z: correction_score(z) > thr)
    if sdim != k:
        raise ValueError(f"reordered Schur form selected {sdim} values, expected {k}")
    return T, Q, k


def krylov_schur(op, s, k, seed, tol=1e-2, max_cycles=20, m=None, complex_arith=False):
    """W (s x keff), T_k (keff x keff) and diagnostics for the operator ``op``.

    ``op`` maps an s-vector to G_hat times it; complex_arith for a complex G_hat.
    """
    info = dict(cycles=0, dense=False, keff=0, ritz=np.zeros(0, dtype=complex))
    if complex_arith:
        return _krylov_schur_complex(op, s, k, seed, tol, max_cycles, m, info)
    if k <= 0 or s == 0:
        return np.zeros((s, 0)), np.zeros((0, 0)), info
    m = 2 * k if m is None else m
    if s <= m:
        G = np.zeros((s, s))
        e = np.zeros(s)
        for i in range(s):
            e[i] = 1.0
            G[:, i] = op(e)
            e[i] = 0.0
        T, Q, keff = schur_wanted(G, k)
        info.update(dense=True, keff=keff, ritz=block_eigs(T)[:keff])
        return Q[:, :keff].copy(), T[:keff, :keff].copy(), info
    v = 2.0 * gemslr_inputs.uniform01(seed, s) - 1.0
    V = np.zeros((s, m + 1))
    Hb = np.zeros((m + 1, m))
    V[:, 0] = v / np.linalg.norm(v)
    p = 0
    for cycle in range(max_cycles):
        info["cycles"] = cycle + 1
        mm = m
        beta = 0.0
        for j in range(p, m):
            w = op(V[:, j])
            wn0 = np.linalg.norm(w)
            h = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h
            h2 = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h2
            h = h + h2
            beta = np.linalg.norm(w)
            Hb[:j + 1, j] = h
            Hb[j + 1, j] = beta
            if beta <= 1e-14 * max(wn0, 1e-300):
                mm = j + 1          # invariant subspace: exact relation
                beta = 0.0
                break
            V[:, j + 1] = w / beta
        Hm = Hb[:mm, :mm]
        T, Q, keff = schur_wanted(Hm, k)
        theta = block_eigs(T)
        resid = np.linalg.norm(beta * Q[mm - 1, :keff])      # residual of the wanted subspace
        ok = resid <= tol * np.min(np.abs(theta[:keff])) or beta == 0.0
        if ok or cycle == max_cycles - 1:
            info.update(keff=keff, ritz=theta[:keff], converged=bool(ok), resid=resid)
            return V[:, :mm] @ Q[:, :keff], T[:keff, :keff].copy(), info
        # thick restart: keep the wanted Schur vectors (Krylov-Schur form)
        Vk = V[:, :mm] @ Q[:, :keff]
        vnext = V[:, mm].copy()
        V[:] = 0.0
        V[:, :keff] = Vk
        V[:, keff] = vnext
        bk = beta * Q[mm - 1, :keff]
        Hb[:] = 0.0
        Hb[:keff, :keff] = T[:keff, :keff]
        Hb[keff, :keff] = bk
        p = keff
    raise AssertionError("unreachable")


def _krylov_schur_complex(op, s, k, seed, tol, max_cycles, m, info):
    """krylov_schur in complex arithmetic (same steps, V^H inner products,
    complex Schur form)."""
    if k <= 0 or s == 0:
        return np.zeros((s, 0), dtype=complex), np.zeros((0, 0), dtype=complex), info
    m = 2 * k if m is None else m
    if s <= m:
        G = np.zeros((s, s), dtype=complex)
        e = np.zeros(s, dtype=complex)
        for i in range(s):
            e[i] = 1.0
            G[:, i] = op(e)
            e[i] = 0.0
        T, Q, keff = schur_wanted_complex(G, k)
        info.update(dense=True, keff=keff, ritz=np.diag(T)[:keff])
        return Q[:, :keff].copy(), T[:keff, :keff].copy(), info
    v = (2.0 * gemslr_inputs.uniform01(seed, s) - 1.0).astype(complex)
    V = np.zeros((s, m + 1), dtype=complex)
    Hb = np.zeros((m + 1, m), dtype=complex)
    V[:, 0] = v / np.linalg.norm(v)
    p = 0
    for cycle in range(max_cycles):
        info["cycles"] = cycle + 1
        mm = m
        beta = 0.0
        for j in range(p, m):
            w = op(V[:, j])
            wn0 = np.linalg.norm(w)
            h = V[:, :j + 1].conj().T @ w
            w = w - V[:, :j + 1] @ h
            h2 = V[:, :j + 1].conj().T @ w
            w = w - V[:, :j + 1] @ h2
            h = h + h2
            beta = np.linalg.norm(w)
            Hb[:j + 1, j] = h
            Hb[j + 1, j] = beta
            if beta <= 1e-14 * max(wn0, 1e-300):
                mm = j + 1
                beta = 0.0
                break
            V[:, j + 1] = w / beta
        Hm = Hb[:mm, :mm]
        T, Q, keff = schur_wanted_complex(Hm, k)
        theta = np.diag(T)
        resid = np.linalg.norm(beta * Q[mm - 1, :keff])
        ok = resid <= tol * np.min(np.abs(theta[:keff])) or beta == 0.0
        if ok or cycle == max_cycles - 1:
            info.update(keff=keff, ritz=theta[:keff], converged=bool(ok), resid=resid)
            return V[:, :mm] @ Q[:, :keff], T[:keff, :keff].copy(), info
        Vk = V[:, :mm] @ Q[:, :keff]
        vnext = V[:, mm].copy()
        V[:] = 0.0
        V[:, :keff] = Vk
        V[:, keff] = vnext
        bk = beta * Q[mm - 1, :keff]
        Hb[:] = 0.0
        Hb[:keff, :keff] = T[:keff, :keff]
        Hb[keff, :keff] = bk
        p = keff
    raise AssertionError("unreachable")


def randomized_schur(op, s, k, seed, oversample=None, power=1):
    """W (s x keff), T_k and diagnostics from a randomized block method instead
    of the thick-restart Arnoldi (Sec. 6 names block and randomized variants
    as future work for the set-up):

      1. Omega: s x b, b = k + oversample (oversample defaults to k), entries
         2u - 1 with u the splitmix64(seed) stream, column after column;
      2. Y = G_hat Omega, then ``power`` times: Q = orth(Y), Y = G_hat Q
         (subspace iteration);
      3. Q = orth(Y) (reduced QR), Z = G_hat Q, Rayleigh quotient B = Q^T Z;
      4. B = U T U^T (real Schur form) with the wanted values leading
         (``schur_wanted``, same ranking and pair rule as the Arnoldi);
         W = Q U[:, :keff], T_k = T[:keff, :keff].

    G_hat W = Z U[:, :keff], so the residual ||G_hat W - W T_k|| is reported
    without further products.  When s <= b the operator is formed densely as
    in ``krylov_schur``."""
    info = dict(dense=False, keff=0, ritz=np.zeros(0, dtype=complex), products=0)
    if k <= 0 or s == 0:
        return np.zeros((s, 0)), np.zeros((0, 0)), info
    b = k + (k if oversample is None else int(oversample))
    if s <= b:
        W, Tk, i2 = krylov_schur(op, s, k, seed, m=b)
        info.update(dense=True, keff=i2["keff"], ritz=i2["ritz"], products=s)
        return W, Tk, info
    u = gemslr_inputs.uniform01(seed, s * b)
    Omega = (2.0 * u - 1.0).reshape(b, s).T

    def apply_block(X):
        info["products"] += X.shape[1]
        return np.column_stack([op(X[:, c]) for c in range(X.shape[1])])

    Y = apply_block(Omega)
    for _ in range(int(power)):
        Q, _ = np.linalg.qr(Y)
        Y = apply_block(Q)
    Q, _ = np.linalg.qr(Y)
    Z = apply_block(Q)
    B = Q.T @ Z
    T, U, keff = schur_wanted(B, k)
    W = Q @ U[:, :keff]
    Tk = T[:keff, :keff].copy()
    resid = np.linalg.norm(Z @ U[:, :keff] - W @ Tk)
    info.update(keff=keff, ritz=block_eigs(T)[:keff], resid=resid)
    return W, Tk, info


def correction_matrix(Tk):
    """H = (I - T_k)^{-1} - I, the k x k middle factor of eq. (gemslr5)."""
    k = Tk.shape[0]
    if k == 0:
        return np.zeros((0, 0), dtype=Tk.dtype)
    I = np.eye(k)
    return np.linalg.solve(I - Tk, I) - I
