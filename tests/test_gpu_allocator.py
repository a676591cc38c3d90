"""Device memory through the caller's allocator (gemslr_options.dev_alloc /
dev_free): the Python binding hands the library PyTorch's caching allocator.
The handle's device bytes must show up in PyTorch's accounting and go back when
the handle is destroyed; results do not depend on the allocator; a failing
allocator gives NOMEM, and a half-given pair is an argument error."""
import ctypes

import numpy as np
import pytest

import gemslr_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problem():
    from paper_2205_03224_gb300 import partition_geometric
    A, xyz = gi.grid_operator((13, 11, 9), beta=0.4)
    return A, partition_geometric(A, xyz, 3, 8)


def test_torch_allocator_accounts_and_releases(torch_cuda):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, part = _problem()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    G = Gemslr(A, part, ilu="ilut", tau=1e-2, lfil=5, rank=5, precision="mixed")
    held = torch.cuda.memory_allocated() - before
    assert held >= G.stats()["device_bytes"] > 0
    r = torch.from_numpy(gi.rhs_uniform(A.n, 3)).cuda()
    z_torch = G.apply(r)
    x, info = G.solve(r, restart=20, rtol=1e-8)
    assert info[0]["converged"]
    G.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() - before < held
    G2 = Gemslr(A, part, ilu="ilut", tau=1e-2, lfil=5, rank=5, precision="mixed", allocator=None)
    assert torch.cuda.memory_allocated() - before < held     # cudaMalloc: outside PyTorch's pool
    assert torch.equal(G2.apply(r), z_torch)


def test_failing_or_half_allocator_is_rejected(torch_cuda):
    from paper_2205_03224_gb300 import _lib
    from paper_2205_03224_gb300.api import options
    A, part = _problem()
    lib = _lib.load()
    keep = []
    csr = _lib.csr_struct(A, keep)
    prt = _lib.partition_struct(part, keep)
    failing = (_lib.ALLOC_FN(lambda n, ctx: None), _lib.FREE_FN(lambda p, ctx: None))
    o = options(ilu="ilu0", rank=2, allocator=failing)
    h = ctypes.c_void_p()
    st = lib.gemslr_setup(ctypes.byref(csr), ctypes.byref(prt), ctypes.byref(o), ctypes.byref(h))
    assert st == 8 and not h.value                         # GEMSLR_ERR_NOMEM
    assert "allocator" in lib.gemslr_last_error().decode()
    o = options(ilu="ilu0", rank=2)
    o.dev_alloc = failing[0]                               # dev_free missing
    st = lib.gemslr_setup(ctypes.byref(csr), ctypes.byref(prt), ctypes.byref(o), ctypes.byref(h))
    assert st == 1 and not h.value
