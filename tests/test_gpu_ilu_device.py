"""ILU(0) of every diagonal block computed on the GPU (set-up, Alg. 1): the
factors must be bit-identical to the host ILU(0), which is checked against
the oracle's ILU(0) in test_gpu_solve, and the solve must be unchanged."""
import numpy as np
import pytest

import gemslr_inputs as gi
from tests.helpers import oracle_hierarchy, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("name", ["c1", "rank0", "tinyparts", "bigblock"])
def test_device_ilu0_equals_host_ilu0(torch_cuda, name):
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    rank = {"c1": 8, "rank0": 0, "tinyparts": 3, "bigblock": 4}[name]
    Gh = Gemslr(A, part, ilu="ilu0", rank=rank)
    Gd = Gemslr(A, part, ilu="ilu0_device", rank=rank)
    fh, fd = Gh.export_factors(), Gd.export_factors()
    pairs = [(a[k], b[k]) for a, b in zip(fh["levels"], fd["levels"]) for k in ("L", "U")]
    pairs += [(fh["last"][k], fd["last"][k]) for k in ("L", "U")]
    for a, b in pairs:
        assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
        assert np.array_equal(a.data, b.data)          # bit-identical
    assert Gh.stats()["nclamp"] == Gd.stats()["nclamp"]


def test_device_ilu0_factors_match_oracle_and_solve(torch_cuda):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem("c1")
    M = oracle_hierarchy("c1")
    G = Gemslr(A, part, ilu="ilu0_device", rank=8)
    f, ref = G.export_factors(), M.factors()
    for lf, rf in zip(f["levels"], ref["levels"]):
        for key in ("L", "U"):
            assert np.array_equal(lf[key].indices, rf[key].indices)
            assert np.allclose(lf[key].data, rf[key].data, rtol=1e-12, atol=0.0)
    b = gi.rhs_uniform(A.n, 2)
    x, info = G.solve(torch.from_numpy(b).cuda(), restart=30, rtol=1e-8)
    res = np.linalg.norm(b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
    assert info[0]["converged"] and res <= 1e-8


def test_device_ilu0_mixed_application_equals_host_ilu0(torch_cuda):
    """Identical factors give the identical mixed-precision application."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem("tinyparts")
    r = torch.from_numpy(gi.rhs_uniform(A.n, 5)).cuda()
    zh = Gemslr(A, part, ilu="ilu0", rank=3, precision="mixed").apply(r)
    zd = Gemslr(A, part, ilu="ilu0_device", rank=3, precision="mixed").apply(r)
    assert torch.equal(zh, zd)
