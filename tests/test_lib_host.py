"""Host-side checks of the C-ABI library (no GPU needed).

The shared library must build for sm_103a, load, and export every entry
point declared in include/gemslr.h.  The partitioner is host logic and must
reproduce the oracle's multilevel ordering exactly (integer work: bit-exact).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import gemslr_inputs as gi
from oracle.partition import multilevel_partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_03224_gb300 import build
    build.build()
    from paper_2205_03224_gb300 import _lib
    return _lib.load()


def test_header_symbols_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "gemslr.h")).read()
    names = sorted(set(re.findall(r"\b(gemslr_[a-z_]+)\s*\(", hdr)))
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_default_options(lib):
    from paper_2205_03224_gb300 import _lib
    o = _lib.Options()
    lib.gemslr_default_options(ctypes.byref(o))
    assert o.ilu_kind == 1 and o.ilut_tau == 1e-3 and o.ilut_lfil == 10
    assert o.arnoldi_tol == 1e-2 and o.arnoldi_max_cycles == 20 and o.precision == 0
    assert o.shift == 0.0 and o.lowrank_method == 0 and o.lowrank_power == 1


@pytest.mark.parametrize("case", [("2d", (32, 32), 0.0, 2, 4), ("3d", (9, 7, 6), 0.3, 3, 4),
                                  ("3d", (12, 10, 11), 0.0, 4, 8), ("3d", (64, 64, 64), 0.1, 4, 64)])
def test_partition_matches_oracle_bit_exact(lib, case):
    from paper_2205_03224_gb300 import partition_geometric
    _, dims, beta, nlev, p = case
    A, xyz = gi.grid_operator(dims, beta=beta)
    ref = multilevel_partition(A.to_scipy(), xyz, nlev, p)
    got = partition_geometric(A, xyz, nlev, p)
    for key in ("perm", "level_ptr", "nblk", "block_ptr"):
        assert np.array_equal(np.asarray(got[key]), np.asarray(ref[key])), key


def test_partition_rejects_bad_arguments(lib):
    from paper_2205_03224_gb300 import partition_geometric
    from paper_2205_03224_gb300._lib import GemslrError
    A, xyz = gi.laplace2d(8)
    with pytest.raises(GemslrError):
        partition_geometric(A, xyz, 3, 3)          # p not a power of two
    with pytest.raises(GemslrError):
        partition_geometric(A, xyz, 1, 4)          # needs a Schur level


def test_binding_argument_counts_match_the_header(lib):
    """Every entry point declared in include/gemslr.h has ctypes argument types
    in the binding, as many as the declaration has parameters."""
    hdr = open(os.path.join(ROOT, "include", "gemslr.h")).read()
    code = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    decls = re.findall(r"\b(gemslr_[a-z_]+)\s*\(([^;{]*?)\)\s*;", code)
    assert len(decls) >= 25
    for name, args in decls:
        args = args.strip()
        nparam = 0 if args in ("", "void") else len(args.split(","))
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == nparam, (name, nparam, len(fn.argtypes))


def test_local_order_and_batch_from_factors_reject_bad_arguments(lib):
    """Argument errors of the host-only entry points are reported before any
    device work: a NULL permutation or an out-of-range first level for the
    local order, NULL factors for the batch set-up from factors."""
    from paper_2205_03224_gb300 import _lib, local_order, partition_geometric
    from paper_2205_03224_gb300._lib import GemslrError
    A, xyz = gi.grid_operator((9, 7, 6), beta=0.3)
    part = partition_geometric(A, xyz, 3, 4)
    with pytest.raises(GemslrError):
        local_order(part, xyz, 4)                  # first level past nlev
    keep = []
    prt = _lib.partition_struct(part, keep)
    st = lib.gemslr_local_order(A.n, _lib.ptr(np.ascontiguousarray(xyz, dtype=np.int32)), ctypes.byref(prt), 1,
                                None)
    assert _lib.STATUS[st] == "ERR_ARG"
    csr = _lib.csr_struct(A, keep)
    h = ctypes.c_void_p()
    st = lib.gemslr_setup_batch_from_factors(1, ctypes.byref(csr), ctypes.byref(prt), None, None, ctypes.byref(h))
    assert _lib.STATUS[st] == "ERR_ARG" and not h.value
    # the identity case: first level = nlev leaves the permutation unchanged
    same = local_order(part, xyz, 3)
    assert np.array_equal(same["perm"], part["perm"])


def test_complex_entry_points_reject_bad_arguments(lib):
    """The complex application and solve report argument errors before any
    device work (NULL handle, NULL vectors, negative nrhs)."""
    from paper_2205_03224_gb300 import _lib
    so = _lib.SolveOpts(30, 100, 1e-8, 0)
    info = (_lib.SolveInfo * 1)()
    assert _lib.STATUS[lib.gemslr_zapply(None, None, None, 1, None)] == "ERR_ARG"
    assert _lib.STATUS[lib.gemslr_zapply(None, None, None, -1, None)] == "ERR_ARG"
    assert _lib.STATUS[lib.gemslr_zfgmres_solve(None, None, None, 1, ctypes.byref(so), info, None)] == "ERR_ARG"
    assert _lib.STATUS[lib.gemslr_zfgmres_solve(None, None, None, 1, None, info, None)] == "ERR_ARG"
