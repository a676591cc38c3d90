"""Restarted flexible GMRES with right preconditioning (Sec. 4.1, Sec. 5 set-up).

Per cycle (Saad 1993, the flexible variant; the paper's outer solver):
  v_1 = r_0 / beta, beta = ||r_0||; for j = 1..m:
     z_j = M^{-1} v_j ; w = A z_j
     modified Gram-Schmidt: h_ij = (w, v_i), w -= h_ij v_i  (i = 1..j)
     h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
     Givens rotations reduce H to triangular form; |g_{j+1}| is the residual
     norm estimate; the cycle stops when |g_{j+1}| <= rtol * ||b||.
  x = x_0 + Z_j y_j with y_j = R_j^{-1} g_{1:j}; r = b - A x (true residual).
Complex arithmetic (``cplx``: a complex preconditioner, e.g. the complex
shift of Sec. 5.2.3, or complex b): inner products h_ij = v_i^H w and the
complex Givens rotation [[conj(c), conj(s)], [-s, c]] with c = h_jj / d,
s = h_{j+1,j} / d, d = sqrt(|h_jj|^2 + h_{j+1,j}^2); for real data these are
the real formulas.  The iterate is then complex; for real A and b the real
part of x has a residual no larger than that of x.
Convergence is declared on the true residual ||b - A x|| <= rtol * ||b||;
otherwise the method restarts from x.  Iterations count inner steps, capped at
``maxit`` (1,000 in the paper: "F").  A happy breakdown
(h_{j+1,j} <= 1e-14 ||A z_j||) ends the cycle.  x_0 = 0.
"""
import numpy as np


def fgmres(A, b, apply_M, restart=50, rtol=1e-8, maxit=1000, x0=None, flexible=True, cplx=False):
    """Returns (x, info) with info = dict(iters, restarts, converged, hist, rel_res_true)."""
    cplx = bool(cplx) or np.iscomplexobj(b)
    dt = np.complex128 if cplx else np.float64
    b = np.asarray(b, dtype=dt)
    n = b.shape[0]
    x = np.zeros(n, dtype=dt) if x0 is None else np.array(x0, dtype=dt)
    bnorm = np.linalg.norm(b)
    hist = []
    its = 0
    restarts = 0
    if bnorm == 0.0:
        return x, dict(iters=0, restarts=0, converged=True, hist=[], rel_res_true=0.0)
    r = b - A @ x
    beta = np.linalg.norm(r)
    converged = beta <= rtol * bnorm
    while not converged and its < maxit:
        m = restart
        V = np.zeros((n, m + 1), dtype=dt)
        Z = np.zeros((n, m), dtype=dt)
        H = np.zeros((m + 1, m), dtype=dt)
        cs = np.zeros(m, dtype=dt)
        sn = np.zeros(m, dtype=dt)
        g = np.zeros(m + 1, dtype=dt)
        g[0] = beta
        V[:, 0] = r / beta
        jdone = 0
        for j in range(m):
            Z[:, j] = apply_M(V[:, j])
            w = A @ Z[:, j]
            its += 1
            wn0 = np.linalg.norm(w)
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[:, i], w) if cplx else V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = abs(H[j + 1, j]) <= 1e-14 * wn0
            if not breakdown:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(abs(H[j, j]), abs(H[j + 1, j]))
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            hist.append(abs(g[j + 1]) / bnorm)
            jdone = j + 1
            if abs(g[j + 1]) <= rtol * bnorm or breakdown or its >= maxit:
                break
        y = np.zeros(jdone, dtype=dt)
        for i in range(jdone - 1, -1, -1):               # R y = g
            y[i] = (g[i] - H[i, i + 1:jdone] @ y[i + 1:]) / H[i, i]
        if flexible:
            x = x + Z[:, :jdone] @ y
        else:
            x = x + apply_M(V[:, :jdone] @ y)
        r = b - A @ x
        beta = np.linalg.norm(r)
        converged = beta <= rtol * bnorm
        if not converged:
            restarts += 1
    return x, dict(iters=its, restarts=restarts, converged=bool(converged), hist=hist,
                   rel_res_true=float(beta / bnorm))
