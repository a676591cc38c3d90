"""GPU parity of M^{-1} (Alg. 2) against the oracle, through the C ABI.

Both sides use the same factors (exported by the oracle, imported by
gemslr_setup_from_factors), so the only differences are rounding: FP64
results must agree to 1e-10 relative (norm-wise) and elementwise to
1e-10 * ||z||_inf.
"""
import numpy as np
import pytest

import gemslr_inputs as gi
from tests.helpers import CASES, oracle_hierarchy, problem, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _lib_from_oracle(name):
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    return Gemslr.from_factors(A, part, M.factors()), M


@pytest.mark.parametrize("name", ["c1", "small3d", "shifted", "rank0", "tinyparts", "bigblock", "c2", "c2local"])
def test_apply_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    G, M = _lib_from_oracle(name)
    n = M.n
    for seed in (11, 12):
        r = gi.rhs_uniform(n, seed)
        z_ref = M.apply(r)
        z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel_err(z, z_ref) <= TOL, name
        assert np.max(np.abs(z - z_ref)) <= TOL * np.max(np.abs(z_ref))


def test_apply_multi_rhs_and_zero(torch_cuda):
    torch = torch_cuda
    G, M = _lib_from_oracle("small3d")
    n = M.n
    R = np.stack([gi.rhs_uniform(n, s) for s in (1, 2, 3)], axis=1)
    Z = G.apply(torch.from_numpy(R).cuda()).cpu().numpy()
    for c in range(3):
        assert rel_err(Z[:, c], M.apply(R[:, c])) <= TOL
    z0 = G.apply(torch.zeros(n, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.all(z0 == 0.0)


def test_tinyparts_has_empty_blocks():
    A, xyz, part = problem("tinyparts")
    bp = part["block_ptr"][: part["nblk"][0] + 1]
    assert np.any(np.diff(bp) == 0)


def test_apply_is_deterministic(torch_cuda):
    torch = torch_cuda
    G, M = _lib_from_oracle("shifted")
    r = torch.from_numpy(gi.rhs_uniform(M.n, 5)).cuda()
    z1 = G.apply(r)
    z2 = G.apply(r)
    assert torch.equal(z1, z2)
