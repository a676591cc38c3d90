"""Python front end of the C ABI (argument marshalling only)."""
import ctypes
import os

import numpy as np

from . import _lib as L


def _stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def partition_geometric(A, coords, nlev, p, p_last=None, local_from=None):
    """Multilevel partition (Alg. 3) computed by the library; returns a dict of arrays.

    local_from: if given, the blocks of levels local_from .. nlev-1 are then put in
    the library's local multicolour order (``local_order``)."""
    lib = L.load()
    keep = []
    csr = L.csr_struct(A, keep)
    n = csr.n
    p_last = p if p_last is None else p_last
    coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(n, 3)
    perm = np.zeros(n, dtype=np.int32)
    level_ptr = np.zeros(nlev + 1, dtype=np.int64)
    nblk = np.zeros(nlev, dtype=np.int32)
    block_ptr = np.zeros((nlev - 1) * (p + 1) + p_last + 1, dtype=np.int64)
    L.check(lib.gemslr_partition_geometric(ctypes.byref(csr), L.ptr(coords), nlev, p, p_last, L.ptr(perm),
                                           L.ptr(level_ptr), L.ptr(nblk), L.ptr(block_ptr)))
    part = dict(perm=perm, level_ptr=level_ptr, nblk=nblk, block_ptr=block_ptr)
    if local_from is not None:
        part = local_order(part, coords, local_from)
    return part


def local_order(part, coords, first_level):
    """The library's local multicolour order inside the blocks of levels first_level on (Sec. 3.2)."""
    lib = L.load()
    keep = []
    n = len(part["perm"])
    coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(n, 3)
    prt = L.partition_struct(part, keep)
    out = np.zeros(n, dtype=np.int32)
    L.check(lib.gemslr_local_order(n, L.ptr(coords), ctypes.byref(prt), int(first_level), L.ptr(out)))
    return dict(part, perm=out)


def torch_allocator():
    """(dev_alloc, dev_free) callbacks that take device memory from PyTorch's
    caching allocator on the current device and stream.  Keep the returned
    objects alive as long as the handle that uses them."""
    import torch

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      torch.cuda.current_stream())
        except Exception:
            return None

    def _free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    return L.ALLOC_FN(_alloc), L.FREE_FN(_free)


def options(ilu="ilut", tau=1e-3, lfil=10, rank=0, precision="fp64", arnoldi_tol=1e-2, max_cycles=20,
            strict_pivots=False, allocator=None, lowrank="arnoldi", power=1, shift=0.0):
    """gemslr_options; allocator: None (cudaMalloc) or a (dev_alloc, dev_free) pair of callbacks;
    lowrank: "arnoldi" or "randomized" set-up of the corrections (power: subspace-iteration passes);
    shift: complex diagonal shift of the factorisations (0: the real method)."""
    o = L.Options()
    L.load().gemslr_default_options(ctypes.byref(o))
    o.ilu_kind = {"ilu0": 0, "ilut": 1, "ilu0_device": 2, "ilut_device": 3}[ilu]
    o.ilut_tau = tau
    o.ilut_lfil = lfil
    ranks = list(rank) if np.ndim(rank) else [int(rank)] * L.MAX_LEVELS
    for i in range(L.MAX_LEVELS):
        o.rank[i] = ranks[i] if i < len(ranks) else 0
    o.precision = {"fp64": 0, "mixed": 1}[precision]
    o.arnoldi_tol = arnoldi_tol
    o.arnoldi_max_cycles = max_cycles
    o.strict_pivots = 1 if strict_pivots else 0
    o.lowrank_method = {"arnoldi": 0, "randomized": 1}[lowrank]
    o.lowrank_power = int(power)
    o.shift = float(shift)
    if allocator is not None:
        o.dev_alloc, o.dev_free = allocator
    return o


def _resolve_allocator(opts):
    """The allocator option: "torch" (default: PyTorch's caching allocator) or None (cudaMalloc)."""
    a = opts.pop("allocator", "torch")
    if a is None:
        return None
    if a == "torch":
        return torch_allocator()
    raise ValueError(f"unknown allocator {a!r}")


def _factors_struct(fac, keep):
    """gemslr_factors view of a factor dict (layout of ``oracle``'s factors()); arrays kept alive in keep.
    Complex factors (the complex shift) pass their imaginary parts separately."""
    lv = fac["levels"]
    arr = (L.LevelFactors * max(len(lv), 1))()
    keep.append(arr)

    def parts(X):
        X = np.asarray(X)
        re = np.asfortranarray(X.real, dtype=np.float64)
        im = np.asfortranarray(X.imag, dtype=np.float64) if np.iscomplexobj(X) else None
        keep.extend([re, im])
        return re, im

    for i, f in enumerate(lv):
        W, Wi = parts(f["W"])
        H, Hi = parts(f["H"])
        Lm, Li = L.mat_struct_z(f["L"], keep)
        Um, Ui = L.mat_struct_z(f["U"], keep)
        arr[i] = L.LevelFactors(Lm, Um, L.mat_struct(f["E"], keep), L.mat_struct(f["F"], keep),
                                W.shape[1], L.ptr(W) if W.size else None, L.ptr(H) if H.size else None,
                                Li, Ui, L.ptr(Wi) if Wi is not None and Wi.size else None,
                                L.ptr(Hi) if Hi is not None and Hi.size else None)
    lL, lLi = L.mat_struct_z(fac["last"]["L"], keep)
    lU, lUi = L.mat_struct_z(fac["last"]["U"], keep)
    return L.Factors(len(lv) + 1, arr, lL, lU, lLi, lUi)


def _is_complex_factors(fac):
    import scipy.sparse as sp
    mats = [f[k] for f in fac["levels"] for k in ("L", "U", "W", "H")] + [fac["last"]["L"], fac["last"]["U"]]
    return any(np.iscomplexobj(m.data if sp.issparse(m) else np.asarray(m)) for m in mats)


class Gemslr:
    """Handle of a GeMSLR preconditioner living on the current CUDA device.

    Device memory comes from PyTorch's caching allocator unless allocator=None
    (then the library calls cudaMalloc itself)."""

    def __init__(self, A, part, _handle=None, _alloc=None, _complex=False, **opts):
        self._lib = L.load()
        self.n = int(len(part["perm"]))
        self.nlev = int(len(part["nblk"]))
        # complex handle (complex shift, Sec. 5.2.3): apply/solve take complex128 tensors
        self.complex = bool(_complex) or float(opts.get("shift", 0.0)) != 0.0
        if _handle is not None:
            self._h = _handle
            self._alloc = _alloc
            return
        keep = []
        csr = L.csr_struct(A, keep)
        prt = L.partition_struct(part, keep)
        self._alloc = _resolve_allocator(opts)
        o = options(allocator=self._alloc, **opts)
        h = ctypes.c_void_p()
        L.check(self._lib.gemslr_setup(ctypes.byref(csr), ctypes.byref(prt), ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_factors(cls, A, part, fac, **opts):
        """Handle built from given factors (dict as produced by ``oracle``'s factors())."""
        lib = L.load()
        keep = []
        csr = L.csr_struct(A, keep)
        prt = L.partition_struct(part, keep)
        fs = _factors_struct(fac, keep)
        alloc = _resolve_allocator(opts)
        o = options(allocator=alloc, **opts)
        h = ctypes.c_void_p()
        L.check(lib.gemslr_setup_from_factors(ctypes.byref(csr), ctypes.byref(prt), ctypes.byref(fs),
                                              ctypes.byref(o), ctypes.byref(h)))
        return cls(A, part, _handle=h, _alloc=alloc, _complex=_is_complex_factors(fac))

    def save_factors(self, path):
        """Write every factor of the handle to `path` (checkpoint of the set-up)."""
        L.check(self._lib.gemslr_save_factors(self._h, os.fsencode(path)))

    @classmethod
    def load_factors(cls, A, part, path, **opts):
        """Handle from a factor file written by save_factors (nothing is factored)."""
        lib = L.load()
        keep = []
        csr = L.csr_struct(A, keep)
        prt = L.partition_struct(part, keep)
        alloc = _resolve_allocator(opts)
        o = options(allocator=alloc, **opts)
        h = ctypes.c_void_p()
        L.check(lib.gemslr_load_factors(ctypes.byref(csr), ctypes.byref(prt), os.fsencode(path), ctypes.byref(o),
                                        ctypes.byref(h)))
        return cls(A, part, _handle=h, _alloc=alloc)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gemslr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, r):
        """z = M^{-1} r for a CUDA float64 tensor r of shape (n,) or (n, nrhs) column-major
        (complex128 for a complex handle)."""
        import torch
        if self.complex:
            r = r.to(torch.complex128)
        r = r.contiguous() if r.dim() == 1 else r.t().contiguous().t()
        z = torch.empty_like(r)
        nrhs = 1 if r.dim() == 1 else r.shape[1]
        fn = self._lib.gemslr_zapply if self.complex else self._lib.gemslr_apply
        L.check(fn(self._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), nrhs, _stream(torch)))
        return z

    def solve(self, b, restart=50, rtol=1e-8, maxit=1000, check=True, ortho="auto"):
        """FGMRES(restart) on A x = b; returns (x, [info dict per right-hand side]).

        ortho: "auto" (delayed reorthogonalisation where M^{-1} is linear) or
        "cgs2" (classical Gram-Schmidt with a selective second pass).  A complex handle solves in
        complex arithmetic (b and x complex128; ortho is ignored)."""
        import torch
        if self.complex:
            b = b.to(torch.complex128)
        b = b.contiguous() if b.dim() == 1 else b.t().contiguous().t()
        x = torch.empty_like(b)
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        so = L.SolveOpts(restart, maxit, rtol, {"auto": 0, "cgs2": 1}[ortho])
        info = (L.SolveInfo * nrhs)()
        fn = self._lib.gemslr_zfgmres_solve if self.complex else self._lib.gemslr_fgmres_solve
        st = fn(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs, ctypes.byref(so), info,
                _stream(torch))
        infos = [dict(iters=i.iters, restarts=i.restarts, converged=bool(i.converged), reorth=i.reorth,
                      rel_res_est=i.rel_res_est, rel_res_true=i.rel_res_true, t_total_ms=i.t_total_ms,
                      status=L.STATUS.get(st, st)) for i in info]
        if check and st not in (0, 4):
            L.check(st)
        return x, infos

    def stats(self):
        out = np.zeros(8 + 6 * self.nlev)
        L.check(self._lib.gemslr_get_stats(self._h, L.ptr(out), len(out)))
        lev = [dict(d=int(out[8 + 6 * l]), s=int(out[9 + 6 * l]), k=int(out[10 + 6 * l]),
                    nnz_lu=int(out[11 + 6 * l]), wavefronts_L=int(out[12 + 6 * l]),
                    wavefronts_U=int(out[13 + 6 * l])) for l in range(self.nlev)]
        return dict(n=int(out[0]), nlev=int(out[1]), nclamp=int(out[2]), nnz_A=int(out[3]),
                    nnz_factors=int(out[4]), bytes_per_apply=float(out[5]), setup_ms=float(out[6]),
                    device_bytes=int(out[7]), levels=lev)

    def set_inner_steps(self, steps):
        """Alg. 2 step 9: `steps` GMRES steps on the root level's inexact Schur
        complement inside every M^{-1} (0 restores the standard application)."""
        L.check(self._lib.gemslr_set_inner_steps(self._h, int(steps)))

    # ---- learned interface correction (an addition to the method) ----
    def learned_train(self, coords, channels=32, npairs=20000, epochs=10, batch=64, lr=1e-3, seed=4):
        """Train the level-l* correction network on the method's own pairs; returns the loss per epoch."""
        coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 3)
        o = L.LearnedOpts(channels, npairs, epochs, batch, lr, seed)
        hist = np.zeros(max(epochs, 1))
        L.check(self._lib.gemslr_learned_train(self._h, L.ptr(coords), ctypes.byref(o), L.ptr(hist)))
        return hist[:epochs]

    def learned_enable(self, on=True):
        L.check(self._lib.gemslr_learned_enable(self._h, 1 if on else 0))

    def learned_info(self):
        out = np.zeros(4)
        L.check(self._lib.gemslr_learned_info(self._h, L.ptr(out)))
        return dict(sites=int(out[0]), channels=int(out[1]), dscale=float(out[2]), nparams=int(out[3]))

    def learned_params(self, params=None):
        n = self.learned_info()["nparams"]
        if params is None:
            out = np.zeros(n)
            L.check(self._lib.gemslr_learned_params(self._h, 1, L.ptr(out), n))
            return out
        params = np.ascontiguousarray(params, dtype=np.float64)
        L.check(self._lib.gemslr_learned_params(self._h, 0, L.ptr(params), n))

    def learned_loss_grad(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        loss = np.zeros(1)
        grad = np.zeros(self.learned_info()["nparams"])
        L.check(self._lib.gemslr_learned_loss_grad(self._h, x.shape[0], L.ptr(x), L.ptr(y), L.ptr(loss), L.ptr(grad)))
        return float(loss[0]), grad

    def export_factors(self):
        """Copy the factors to host (dict with the layout of ``from_factors``)."""
        import scipy.sparse as sp
        nl = self.nlev
        counts = np.zeros(4 + 9 * (nl - 1), dtype=np.int64)
        L.check(self._lib.gemslr_factor_sizes(self._h, L.ptr(counts), len(counts)))
        keep = []

        cx = self.complex

        def mk(nrows, ncols, nnz):
            rp = np.zeros(nrows + 1, dtype=np.int64)
            ci = np.zeros(max(nnz, 1), dtype=np.int32)
            v = np.zeros(max(nnz, 1), dtype=np.float64)
            vi = np.zeros(max(nnz, 1), dtype=np.float64)
            keep.append((rp, ci, v, nrows, ncols, nnz, vi))
            return L.Mat(nrows, ncols, L.ptr(rp), L.ptr(ci), L.ptr(v)), len(keep) - 1

        def im(i):
            return L.ptr(keep[i][6]) if cx else None

        arr = (L.LevelFactors * max(nl - 1, 1))()
        meta = []
        for l in range(nl - 1):
            c = counts[1 + 9 * l: 10 + 9 * l]
            nL, nU, nE, nF, k, d, s = [int(t) for t in c[:7]]
            mL, iL = mk(d, d, nL)
            mU, iU = mk(d, d, nU)
            mE, iE = mk(s, d, nE)
            mF, iF = mk(d, s, nF)
            W = np.zeros((s, max(k, 1)), dtype=np.float64, order="F")
            H = np.zeros((max(k, 1), max(k, 1)), dtype=np.float64, order="F")
            Wi = np.zeros_like(W)
            Hi = np.zeros_like(H)
            arr[l] = L.LevelFactors(mL, mU, mE, mF, k, L.ptr(W), L.ptr(H), im(iL), im(iU),
                                    L.ptr(Wi) if cx else None, L.ptr(Hi) if cx else None)
            meta.append((iL, iU, iE, iF, W, H, Wi, Hi, k, int(c[7]), int(c[8])))
        c = counts[1 + 9 * (nl - 1):]
        nLl, nUl, sl = int(c[0]), int(c[1]), int(c[2])
        mLl, iLl = mk(sl, sl, nLl)
        mUl, iUl = mk(sl, sl, nUl)
        fs = L.Factors(nl, arr, mLl, mUl, im(iLl), im(iUl))
        L.check(self._lib.gemslr_export_factors(self._h, ctypes.byref(fs)))

        def tocsr(i, imag=False):
            rp, ci, v, nr, nc, nnz, vi = keep[i]
            vals = v[:nnz] + 1j * vi[:nnz] if imag and cx else v[:nnz]
            return sp.csr_matrix((vals, ci[:nnz], rp), shape=(nr, nc))

        def dense(X, Xi, r, c):
            return np.array(X[:r, :c] + 1j * Xi[:r, :c]) if cx else np.array(X[:r, :c])

        levels = []
        for (iL, iU, iE, iF, W, H, Wi, Hi, k, s0, e0) in meta:
            levels.append(dict(s=s0, e=e0, L=tocsr(iL, True), U=tocsr(iU, True), E=tocsr(iE), F=tocsr(iF),
                               W=dense(W, Wi, W.shape[0], k), H=dense(H, Hi, k, k)))
        return dict(levels=levels, last=dict(L=tocsr(iLl, True), U=tocsr(iUl, True)))


class GemslrBatch:
    """Many independent systems solved together (up to 8 right-hand sides each)."""

    MAX_RHS = 8

    def __init__(self, As, parts, **opts):
        self._lib = L.load()
        keep = []
        n = len(As)
        csrs = (L.CSR * n)(*[L.csr_struct(A, keep) for A in As])
        prts = (L.Partition * n)(*[L.partition_struct(p, keep) for p in parts])
        self._alloc = _resolve_allocator(opts)
        o = options(allocator=self._alloc, **opts)
        h = ctypes.c_void_p()
        L.check(self._lib.gemslr_setup_batch(n, csrs, prts, ctypes.byref(o), ctypes.byref(h)), batch=True)
        self._h = h
        self.sizes = [int(c.n) for c in csrs]
        self.nsys = n

    @classmethod
    def from_factors(cls, As, parts, facs, **opts):
        """Batch built from given factors, one dict per system (layout of ``oracle``'s factors())."""
        self = cls.__new__(cls)
        self._lib = L.load()
        keep = []
        n = len(As)
        csrs = (L.CSR * n)(*[L.csr_struct(A, keep) for A in As])
        prts = (L.Partition * n)(*[L.partition_struct(p, keep) for p in parts])
        fss = (L.Factors * n)(*[_factors_struct(f, keep) for f in facs])
        self._alloc = _resolve_allocator(opts)
        o = options(allocator=self._alloc, **opts)
        h = ctypes.c_void_p()
        L.check(self._lib.gemslr_setup_batch_from_factors(n, csrs, prts, fss, ctypes.byref(o), ctypes.byref(h)),
                batch=True)
        self._h = h
        self.sizes = [int(c.n) for c in csrs]
        self.nsys = n
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gemslr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, r, nrhs):
        """z = M_s^{-1} r for the concatenated column-major blocks of every system."""
        import torch
        r = r.contiguous()
        z = torch.empty_like(r)
        L.check(self._lib.gemslr_batch_apply(self._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                             nrhs, _stream(torch)), batch=True)
        return z

    def solve(self, b, nrhs, restart=50, rtol=1e-8, maxit=1000, check=True):
        import torch
        b = b.contiguous()
        x = torch.empty_like(b)
        so = L.SolveOpts(restart, maxit, rtol, 0)
        info = (L.SolveInfo * (self.nsys * nrhs))()
        st = self._lib.gemslr_batch_fgmres_solve(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                                 nrhs, ctypes.byref(so), info, _stream(torch))
        infos = [dict(iters=i.iters, restarts=i.restarts, converged=bool(i.converged),
                      rel_res_true=i.rel_res_true, t_total_ms=i.t_total_ms, status=L.STATUS.get(st, st)) for i in info]
        if check and st not in (0, 4):
            L.check(st, batch=True)
        return x, infos

    def stats(self):
        out = np.zeros(13)
        L.check(self._lib.gemslr_batch_stats(self._h, L.ptr(out), 13), batch=True)
        return dict(nsys=int(out[0]), rows=int(out[1]), nnz_factors=int(out[2]), bytes_per_apply=float(out[3]),
                    setup_ms=float(out[4]), tune_ms=float(out[5]), rows_couple=int(out[6]), rows_krylov=int(out[7]),
                    rhs_per_cta=int(out[8]), lev0_rows=int(out[9]), lev0_l_bytes=int(out[10]),
                    lev0_u_bytes=int(out[11]), lev0_f_nnz=int(out[12]))
