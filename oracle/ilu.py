"""Incomplete LU of one diagonal block and the triangular substitutions.

Sec. 2.1/2.4 and Alg. 1: B_l^{-1} is applied as (L_l U_l)^{-1} with L_l U_l an
incomplete factorisation of each diagonal block B_l^{(j)}.  The loops live in
oracle/c/oracle_ilu.c (real) and oracle/c/oracle_ilu_z.c (complex: the
complex-shifted blocks of Sec. 5.2.3); this module converts to and from scipy
CSR and picks the complex loops for complex matrices and vectors.
"""
import ctypes

import numpy as np
import scipy.sparse as sp

from ._clib import lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr_parts(B):
    B = sp.csr_matrix(B)
    B.sort_indices()
    rp = np.ascontiguousarray(B.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(B.indices, dtype=np.int32)
    cplx = np.iscomplexobj(B.data)
    v = np.ascontiguousarray(B.data, dtype=np.complex128 if cplx else np.float64)
    return B.shape[0], rp, ci, v


def _unpack(fp, cplx=False):
    f = fp.contents
    n = f.n
    lrp = np.ctypeslib.as_array(f.lrp, shape=(n + 1,)).copy()
    urp = np.ctypeslib.as_array(f.urp, shape=(n + 1,)).copy()
    nl, nu = int(lrp[-1]), int(urp[-1])
    w = 2 if cplx else 1
    lci = np.ctypeslib.as_array(f.lci, shape=(max(nl, 1),))[:nl].copy()
    lv = np.ctypeslib.as_array(f.lv, shape=(max(w * nl, 1),))[:w * nl].copy()
    uci = np.ctypeslib.as_array(f.uci, shape=(max(nu, 1),))[:nu].copy()
    uv = np.ctypeslib.as_array(f.uv, shape=(max(w * nu, 1),))[:w * nu].copy()
    if cplx:
        lv, uv = lv.view(np.complex128), uv.view(np.complex128)
    nclamp = int(f.nclamp)
    (lib().oracle_free_factors_z if cplx else lib().oracle_free_factors)(fp)
    L = sp.csr_matrix((lv, lci, lrp), shape=(n, n))
    U = sp.csr_matrix((uv, uci, urp), shape=(n, n))
    return L, U, nclamp


def ilu0(B):
    """ILU(0) of B: returns (L strictly lower, U upper with diagonal, #clamped pivots)."""
    n, rp, ci, v = _csr_parts(B)
    if n == 0:
        z = sp.csr_matrix((0, 0))
        return z, z, 0
    if np.iscomplexobj(v):
        return _unpack(lib().oracle_ilu0_z(n, _ptr(rp), _ptr(ci), _ptr(v)), cplx=True)
    return _unpack(lib().oracle_ilu0(n, _ptr(rp), _ptr(ci), _ptr(v)))


def ilut(B, tau, lfil):
    """ILUT(tau, lfil) of B (lfil < 0 keeps every entry above the threshold)."""
    n, rp, ci, v = _csr_parts(B)
    if n == 0:
        z = sp.csr_matrix((0, 0))
        return z, z, 0
    if np.iscomplexobj(v):
        return _unpack(lib().oracle_ilut_z(n, _ptr(rp), _ptr(ci), _ptr(v), float(tau), int(lfil)), cplx=True)
    return _unpack(lib().oracle_ilut(n, _ptr(rp), _ptr(ci), _ptr(v), float(tau), int(lfil)))


def lu_solve(L, U, b):
    """x = U^{-1} L^{-1} b, row by row in plain C (L unit lower, U upper); complex
    when the factors or b are."""
    n = L.shape[0]
    cplx = np.iscomplexobj(L.data) or np.iscomplexobj(U.data) or np.iscomplexobj(b)
    dt = np.complex128 if cplx else np.float64
    b = np.ascontiguousarray(b, dtype=dt)
    if n == 0:
        return b.copy()
    y = np.empty(n, dtype=dt)
    x = np.empty(n, dtype=dt)
    ls, us = (lib().oracle_lsolve_z, lib().oracle_usolve_z) if cplx else (lib().oracle_lsolve, lib().oracle_usolve)
    ls(n, _ptr(L.indptr.astype(np.int64)), _ptr(L.indices.astype(np.int32)),
       _ptr(np.ascontiguousarray(L.data, dtype=dt)), _ptr(b), _ptr(y))
    us(n, _ptr(U.indptr.astype(np.int64)), _ptr(U.indices.astype(np.int32)),
       _ptr(np.ascontiguousarray(U.data, dtype=dt)), _ptr(y), _ptr(x))
    return x
