"""GeMSLR setup (Alg. 1) and standard solve (Alg. 2), FP64, plain and slow.

Level structure (reading of "l_ev levels", Sec. 2.4 and Alg. 2's commented
last-level branch): levels l = 0 .. nlev-2 are Schur levels, each with its
B_l (p diagonal blocks, incomplete LU), coupling blocks E_l, F_l and a rank-k
correction W_l, H_l; the last level is the matrix C_{nlev-2} itself, applied
by block-Jacobi incomplete LU over its p_last diagonal blocks with the
off-block entries discarded (Sec. 4.3), and no low-rank term.

Vectors handled by ``apply_perm`` are in the multilevel (permuted) order
x_hat = P^T x, i.e. x_hat[i] = x[perm[i]]; level l owns the contiguous range
[level_ptr[l], level_ptr[l+1]) and A_l acts on the tail [level_ptr[l], n).
"""
import numpy as np
import scipy.sparse as sp

from . import ilu as _ilu
from .lowrank import correction_matrix, krylov_schur, randomized_schur
from .partition import level_blocks


def _factor_blocks(B, bp, kind, tau, lfil, alpha=0.0):
    """Incomplete LU of every diagonal block of B (of B_j + i alpha I when
    alpha != 0, the complex shift of Sec. 5.2.3); block-diagonal L, U."""
    Ls, Us = [], []
    nclamp = 0
    for j in range(len(bp) - 1):
        a, b = bp[j], bp[j + 1]
        Bj = B[a:b, a:b]
        if alpha != 0.0:
            Bj = sp.csr_matrix(Bj, dtype=complex) + 1j * alpha * sp.eye(b - a, format="csr")
        if kind == "ilu0":
            L, U, c = _ilu.ilu0(Bj)
        elif kind == "ilut":
            L, U, c = _ilu.ilut(Bj, tau, lfil)
        elif kind == "exact":
            L, U, c = _ilu.ilut(Bj, 0.0, -1)
        else:
            raise ValueError(kind)
        Ls.append(sp.csr_matrix(L, shape=(b - a, b - a)))
        Us.append(sp.csr_matrix(U, shape=(b - a, b - a)))
        nclamp += c
    n = B.shape[0]
    if n == 0:
        z = sp.csr_matrix((0, 0))
        return z, z, nclamp
    L = sp.block_diag(Ls, format="csr") if Ls else sp.csr_matrix((n, n))
    U = sp.block_diag(Us, format="csr") if Us else sp.csr_matrix((n, n))
    L.sort_indices()
    U.sort_indices()
    return sp.csr_matrix(L, shape=(n, n)), sp.csr_matrix(U, shape=(n, n)), nclamp


class OracleGemslr:
    """Multilevel GeMSLR preconditioner built by the oracle.

    Parameters
    ----------
    A : scipy sparse (n x n)
    part : dict from ``multilevel_partition``
    ilu : "ilu0" | "ilut" | "exact" (ILUT with tau = 0 and no fill limit)
    rank : int or list (per Schur level); 0 disables the correction
    last_ilu : factor kind of the last-level blocks (defaults to ``ilu``)
    inner_steps : Alg. 2 step 9; 0 applies the standard recursion at level 0,
        k > 0 solves S_hat_0 y2 = z2 there by k steps of right-preconditioned
        GMRES (``inner_gmres``)
    shift : complex diagonal shift of the incomplete factorisations (Sec. 5.2.3):
        every diagonal block of every B_l and of the last level is factored
        as B + i alpha I with alpha = shift * sum_i |a_ii| / n (the paper uses
        shift = 0.05); E, F and C are not shifted.  With shift != 0 the
        factors, W, H and every vector of the application are complex, and
        the correction is W H W^H (Sec. 2.2).
    lowrank : "arnoldi" (thick-restart Krylov-Schur, the default) or
        "randomized" (``randomized_schur``: subspace iteration on a random
        block with ``power`` passes, Sec. 6); False skips the corrections.

    Attribute ``stage`` (default None): an extra correction of the deepest
    Schur level l* = nlev - 2, a callable (z2, y2) -> y2' applied after y2 is
    computed there and before the back-substitution with F (the learned
    interface correction, ``oracle.learned.interface_stage``; not in the
    paper: FGMRES tolerates a preconditioner that varies, Sec. 4.1).
    """

    def __init__(self, A, part, ilu="ilu0", tau=1e-3, lfil=10, rank=8, last_ilu=None,
                 arnoldi_tol=1e-2, max_cycles=20, lowrank=True, inner_steps=0, shift=0.0, power=1):
        self.inner_steps = int(inner_steps)
        self.stage = None
        A = sp.csr_matrix(A)
        self.shift = float(shift)
        self.alpha = self.shift * float(np.abs(A.diagonal()).sum()) / A.shape[0] if A.shape[0] else 0.0
        self.n = A.shape[0]
        self.part = part
        self.perm = np.asarray(part["perm"], dtype=np.int64)
        self.nlev = len(part["nblk"])
        Ah = A[self.perm][:, self.perm].tocsr()
        Ah.sort_indices()
        self.Ahat = Ah
        nsch = self.nlev - 1
        ranks = list(rank) if np.ndim(rank) else [int(rank)] * nsch
        self.levels = []
        self.nclamp = 0
        for l in range(nsch):
            s, e, bp = level_blocks(part, l)
            bp = bp - s
            B = Ah[s:e, s:e]
            L, U, c = _factor_blocks(B, bp, ilu, tau, lfil, self.alpha)
            self.nclamp += c
            self.levels.append(dict(s=s, e=e, bp=bp, L=L, U=U,
                                    E=Ah[e:, s:e].tocsr(), F=Ah[s:e, e:].tocsr(),
                                    W=np.zeros((self.n - e, 0)), H=np.zeros((0, 0)),
                                    rank=ranks[l], info=None))
        s, e, bp = level_blocks(part, self.nlev - 1)
        bp = bp - s
        C = Ah[s:, s:].tocsr()
        # block-Jacobi: keep the diagonal blocks only
        keep = sp.block_diag([C[bp[j]:bp[j + 1], bp[j]:bp[j + 1]] for j in range(len(bp) - 1)],
                             format="csr") if C.shape[0] else sp.csr_matrix((0, 0))
        self.last_s = s
        self.last_bp = bp
        self.last_C = keep
        Lc, Uc, c = _factor_blocks(keep, bp, last_ilu or ilu, tau, lfil, self.alpha)
        self.nclamp += c
        self.last_L, self.last_U = Lc, Uc
        self.lowrank_method = "randomized" if lowrank == "randomized" else "arnoldi"
        self.power = int(power)
        if lowrank:
            # bottom-up (Sec. 4.2): level l needs the apply of every level > l
            for l in range(nsch - 1, -1, -1):
                self.build_lowrank(l, arnoldi_tol, max_cycles)

    @classmethod
    def from_factors(cls, A, part, fac):
        """A hierarchy whose factors are given, in the layout of ``factors()``
        (L, U, E, F, W, H per Schur level, L, U of the last level): nothing is
        factored, so Alg. 2 can be applied to factors computed elsewhere (the
        permutation and the level slices still come from A and the partition)."""
        self = cls.__new__(cls)
        self.inner_steps = 0
        self.stage = None
        A = sp.csr_matrix(A)
        self.n = A.shape[0]
        self.part = part
        self.perm = np.asarray(part["perm"], dtype=np.int64)
        self.nlev = len(part["nblk"])
        Ah = A[self.perm][:, self.perm].tocsr()
        Ah.sort_indices()
        self.Ahat = Ah
        cplx = any(np.iscomplexobj(f[k].data if sp.issparse(f[k]) else np.asarray(f[k]))
                   for f in fac["levels"] for k in ("L", "U", "W", "H"))
        self.shift = 0.0
        self.alpha = 1.0 if cplx else 0.0      # only its being nonzero matters (complex arithmetic)
        self.levels = []
        self.nclamp = 0
        for l, f in enumerate(fac["levels"]):
            s, e, bp = level_blocks(part, l)
            W = np.asarray(f["W"])
            self.levels.append(dict(s=s, e=e, bp=bp - s, L=sp.csr_matrix(f["L"]), U=sp.csr_matrix(f["U"]),
                                    E=Ah[e:, s:e].tocsr(), F=Ah[s:e, e:].tocsr(), W=W,
                                    H=np.asarray(f["H"]), rank=W.shape[1], info=None))
        s, e, bp = level_blocks(part, self.nlev - 1)
        self.last_s = s
        self.last_bp = bp - s
        self.last_C = None
        self.last_L = sp.csr_matrix(fac["last"]["L"])
        self.last_U = sp.csr_matrix(fac["last"]["U"])
        self.lowrank_method = "given"
        self.power = 1
        return self

    # ---- pieces of Alg. 2 -------------------------------------------------
    def solve_level(self, r, l):
        """pGeMSLRSolve(r, l) on the tail vector r (length n - level_ptr[l])."""
        if l == self.nlev - 1:
            return _ilu.lu_solve(self.last_L, self.last_U, r)
        lv = self.levels[l]
        d = lv["e"] - lv["s"]
        b1, b2 = r[:d], r[d:]
        z1 = _ilu.lu_solve(lv["L"], lv["U"], b1)                 # z1 = U^-1 L^-1 b1
        z2 = b2 - lv["E"] @ z1                                   # z2 = b2 - E z1
        if l == 0 and self.inner_steps > 0:
            y2 = self.inner_gmres(z2, self.inner_steps)          # S_hat_0 y2 = z2 by GMRES
        else:
            y2 = self.precond_schur(z2, l)                       # y2 = Solve(z2 + u2, l+1)
        if self.stage is not None and l == self.nlev - 2:
            y2 = self.stage(z2, y2)                              # learned correction at l*
        y1 = z1 - _ilu.lu_solve(lv["L"], lv["U"], lv["F"] @ y2)  # y1 = z1 - U^-1 L^-1 F y2
        return np.concatenate([y1, y2])

    def precond_schur(self, z2, l):
        """eq. gemslr6 at level l: C_l^-1 (z2 + W_l H_l W_l^T z2), C_l^-1 the levels below."""
        lv = self.levels[l]
        W, H = lv["W"], lv["H"]
        u2 = W @ (H @ (W.conj().T @ z2)) if W.shape[1] else np.zeros_like(z2)
        return self.solve_level(u2 + z2, l + 1)

    def s_hat(self, v, l):
        """Inexact Schur complement S_hat_l v = C_l v - E_l U_l^-1 L_l^-1 F_l v (Sec. 2.4)."""
        lv = self.levels[l]
        C = self.Ahat[lv["e"]:, lv["e"]:]
        return C @ v - lv["E"] @ _ilu.lu_solve(lv["L"], lv["U"], lv["F"] @ v)

    def inner_gmres(self, z2, k, l=0):
        """Alg. 2 step 9: k steps of GMRES on S_hat_l y = z2 from y = 0, right
        preconditioned by ``precond_schur`` (eq. gemslr6).  Arnoldi with modified
        Gram-Schmidt on the vectors v_j; y = sum_j c_j M_S^-1 v_j with c the
        minimiser of ||beta e_1 - H c|| over the (j+1) x j Hessenberg matrix.
        A happy breakdown (h_{j+1,j} <= 1e-14 ||S_hat M_S^-1 v_j||) ends the
        steps early with the exact solution of the projected problem."""
        beta = np.linalg.norm(z2)
        if beta == 0.0:
            return np.zeros_like(z2)
        V = [z2 / beta]
        Z = []
        H = np.zeros((k + 1, k))
        steps = 0
        for j in range(k):
            Z.append(self.precond_schur(V[j], l))
            w = self.s_hat(Z[j], l)
            w0 = np.linalg.norm(w)
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            steps = j + 1
            if H[j + 1, j] <= 1e-14 * w0:
                break
            V.append(w / H[j + 1, j])
        rhs = np.zeros(steps + 1)
        rhs[0] = beta
        c = np.linalg.lstsq(H[:steps + 1, :steps], rhs, rcond=None)[0]
        return np.column_stack(Z) @ c

    def apply_perm(self, r_hat):
        """M^{-1} in the multilevel ordering."""
        r_hat = np.asarray(r_hat)
        dt = np.complex128 if (self.alpha != 0.0 or np.iscomplexobj(r_hat)) else np.float64
        return self.solve_level(r_hat.astype(dt), 0)

    def apply(self, r):
        """M^{-1} r in the original ordering: P (M_hat^{-1} (P^T r))."""
        y = self.apply_perm(np.asarray(r)[self.perm])
        out = np.empty_like(y)
        out[self.perm] = y
        return out

    def g_hat(self, l, z):
        """G_hat_l z = E_l U_l^-1 L_l^-1 F_l C_l^-1 z with C_l^-1 the apply of levels > l."""
        lv = self.levels[l]
        y = self.solve_level(z, l + 1)
        return lv["E"] @ _ilu.lu_solve(lv["L"], lv["U"], lv["F"] @ y)

    def build_lowrank(self, l, tol=1e-2, max_cycles=20):
        lv = self.levels[l]
        s = self.n - lv["e"]
        if self.lowrank_method == "randomized":
            if self.alpha != 0.0:
                raise ValueError("the randomized set-up is real only")
            W, Tk, info = randomized_schur(lambda z: self.g_hat(l, z), s, lv["rank"], 1000 + l, power=self.power)
        else:
            W, Tk, info = krylov_schur(lambda z: self.g_hat(l, z), s, lv["rank"], 1000 + l,
                                       tol=tol, max_cycles=max_cycles, complex_arith=self.alpha != 0.0)
        lv["W"] = W
        lv["T"] = Tk
        lv["H"] = correction_matrix(Tk)
        lv["info"] = info

    # ---- export -------------------------------------------------------------
    def factors(self):
        """Everything the solve phase reads, in the multilevel ordering."""
        out = dict(n=self.n, perm=self.perm.astype(np.int32), nlev=self.nlev, levels=[])
        for lv in self.levels:
            out["levels"].append(dict(s=lv["s"], e=lv["e"], bp=lv["bp"], L=lv["L"], U=lv["U"],
                                      E=lv["E"], F=lv["F"], W=lv["W"], H=lv["H"]))
        out["last"] = dict(s=self.last_s, bp=self.last_bp, L=self.last_L, U=self.last_U)
        return out
