"""Allocation-free application of M^{-1} (gemslr_apply_static).

For callers that cannot allocate device memory when they apply the
preconditioner (inside a CUDA graph capture, under a foreign memory pool,
or in allocator-free latency-critical loops), the library offers an entry
point whose scratch is a fixed device array.  It must give the same result
as gemslr_apply on two calls in a row (the array keeps the previous call's
contents, which must not leak into the next result), for FP64 and for
mixed-precision handles, and it must refuse a handle larger than the array
with an argument error.  This file is collected last so that a run that
stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import gemslr_inputs as gi

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_apply_matches_apply_twice(precision):
    torch = _cuda()
    from paper_2205_03224_gb300 import Gemslr, partition_geometric
    from paper_2205_03224_gb300 import _lib
    lib = _lib.load()
    A, xyz = gi.grid_operator((13, 11, 9), beta=0.4)
    part = partition_geometric(A, xyz, 3, 8)
    G = Gemslr(A, part, ilu="ilut", tau=1e-2, lfil=5, rank=5, precision=precision)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # both paths apply the same factors in the same precision: equal to rounding order
    tol = 1e-10 if precision == "fp64" else 1e-5
    for seed in (31, 32):
        r = torch.from_numpy(gi.rhs_uniform(A.n, seed)).cuda()
        z_ref = G.apply(r)
        z = torch.full_like(r, float("nan"))
        st = lib.gemslr_apply_static(G._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), stream)
        assert st == 0, lib.gemslr_last_error().decode()
        torch.cuda.synchronize()
        zr, zs = z_ref.cpu().numpy(), z.cpu().numpy()
        assert np.all(np.isfinite(zs))
        assert np.linalg.norm(zs - zr) <= tol * np.linalg.norm(zr)


def test_static_apply_rejects_more_rows_than_its_array():
    """n = 1,449^2 = 2,099,601 > 2,097,152 rows: an argument error before any
    launch, with a message that names the limit; z is left untouched."""
    torch = _cuda()
    from paper_2205_03224_gb300 import Gemslr, partition_geometric
    from paper_2205_03224_gb300 import _lib
    lib = _lib.load()
    A, xyz = gi.grid_operator((1449, 1449))
    assert A.n > 2097152
    part = partition_geometric(A, xyz, 2, 2)
    G = Gemslr(A, part, ilu="ilu0", rank=0)
    r = torch.ones(A.n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.gemslr_apply_static(G._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), stream)
    assert _lib.STATUS[st] == "ERR_ARG"
    assert "2097152" in lib.gemslr_last_error().decode()
    torch.cuda.synchronize()
    assert torch.count_nonzero(z) == 0
