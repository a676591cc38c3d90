"""Mixed-precision M^{-1} (FP32 factors and vectors, BF16 W with FP32
accumulation; FGMRES in FP64): error against the FP64 oracle, and FGMRES
still reaching 1e-8 with the same factors."""
import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import fgmres
from tests.helpers import oracle_hierarchy, problem, rel_err

pytestmark = pytest.mark.gpu

# BF16 keeps 8 significant bits of W: the correction term carries ~4e-3
# relative error, the FP32 substitutions ~1e-6; the bound covers both.
MIXED_TOL = 2e-2


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("name", ["c1", "small3d", "shifted", "c2", "c2local"])
def test_mixed_apply_error_against_fp64_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    G = Gemslr.from_factors(A, part, M.factors(), precision="mixed")
    r = gi.rhs_uniform(M.n, 21)
    z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    err = rel_err(z, M.apply(r))
    assert err <= MIXED_TOL, err
    assert err > 0.0          # it really ran in reduced precision


@pytest.mark.parametrize("name", ["c1", "small3d", "shifted"])
def test_mixed_apply_with_bf16_w_is_fp32_accurate(torch_cuda, name):
    """With W rounded to BF16 on both sides the mixed application differs
    from the FP64 oracle by FP32 rounding only (about 1e-6 relative)."""
    torch = torch_cuda
    from oracle import OracleGemslr
    from paper_2205_03224_gb300 import Gemslr
    from tests.helpers import CASES, round_w_to_bf16
    dims, beta, sigma, nlev, p, ilu, tau, lfil, rank = CASES[name]
    A, xyz, part = problem(name)
    M = OracleGemslr(A.to_scipy(), part, ilu=ilu, tau=tau, lfil=lfil, rank=rank)
    G = Gemslr.from_factors(A, part, round_w_to_bf16(M), precision="mixed")
    r = gi.rhs_uniform(M.n, 22)
    err = rel_err(G.apply(torch.from_numpy(r).cuda()).cpu().numpy(), M.apply(r))
    assert 0.0 < err <= 1e-4, err


@pytest.mark.parametrize("name", ["c1", "small3d", "c2", "c2local"])
def test_mixed_fgmres_reaches_1e8(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    restart = {"c1": 30, "small3d": 20, "c2": 50, "c2local": 50}[name]
    b = gi.rhs_uniform(M.n, 1)
    _, info_ref = fgmres(A.to_scipy(), b, M.apply, restart=restart, rtol=1e-8)
    G = Gemslr.from_factors(A, part, M.factors(), precision="mixed")
    x, info = G.solve(torch.from_numpy(b).cuda(), restart=restart, rtol=1e-8)
    x = x.cpu().numpy()
    res = np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b)
    assert info[0]["converged"] and res <= 1e-8
    assert info[0]["iters"] <= info_ref["iters"] + 3
