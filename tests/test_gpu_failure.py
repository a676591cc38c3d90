"""Failure detection without a GPU fault: the bounded device waits give up and
report GEMSLR_ERR_TIMEOUT, and the CUDA context stays usable."""
import numpy as np
import pytest

import gemslr_inputs as gi
from tests.helpers import oracle_hierarchy, problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_bounded_waits_expire_and_context_survives(torch_cuda):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr, _lib
    # about 1 ms at the SM clock: a wait on an mbarrier that nothing completes
    assert _lib.selftest_wait(2_000_000) == "ERR_TIMEOUT"
    assert "expired" in _lib.load().gemslr_last_error().decode()
    # the context is intact: a normal application still matches the oracle
    A, xyz, part = problem("c1")
    M = oracle_hierarchy("c1")
    G = Gemslr.from_factors(A, part, M.factors())
    r = gi.rhs_uniform(M.n, 3)
    z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_err(z, M.apply(r)) <= 1e-10


def test_selftest_rejects_bad_argument(torch_cuda):
    from paper_2205_03224_gb300 import _lib
    assert _lib.selftest_wait(0) == "ERR_ARG"
