"""Allocation-free application of M^{-1} (gemslr_apply_static).

For callers that cannot allocate device memory when they apply the
preconditioner (inside a CUDA graph capture, under a foreign memory pool,
or in allocator-free latency-critical loops), the library offers an entry
point whose scratch is a fixed device array.  It must give the same result
as gemslr_apply on two calls in a row (the array keeps the previous call's
contents, which must not leak into the next result).  This file is collected
last so that a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import gemslr_inputs as gi

pytestmark = pytest.mark.gpu


def test_static_apply_matches_apply_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_03224_gb300 import Gemslr, partition_geometric
    from paper_2205_03224_gb300 import _lib
    lib = _lib.load()
    A, xyz = gi.grid_operator((13, 11, 9), beta=0.4)
    part = partition_geometric(A, xyz, 3, 8)
    G = Gemslr(A, part, ilu="ilut", tau=1e-2, lfil=5, rank=5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (31, 32):
        r = torch.from_numpy(gi.rhs_uniform(A.n, seed)).cuda()
        z_ref = G.apply(r)
        z = torch.full_like(r, float("nan"))
        st = lib.gemslr_apply_static(G._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), stream)
        assert st == 0, lib.gemslr_last_error().decode()
        torch.cuda.synchronize()
        zr, zs = z_ref.cpu().numpy(), z.cpu().numpy()
        assert np.all(np.isfinite(zs))
        assert np.linalg.norm(zs - zr) <= 1e-10 * np.linalg.norm(zr)
