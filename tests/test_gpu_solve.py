"""GPU FGMRES (Sec. 4.1) and the library's own setup against the oracle."""
import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import fgmres
from tests.helpers import lib_opts, oracle_hierarchy, problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


RESTART = {"c1": 30, "small3d": 20, "shifted": 30, "c2": 50}


@pytest.mark.parametrize("name", ["c1", "small3d", "shifted", "c2"])
def test_fgmres_matches_oracle_iterations(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    b = gi.rhs_uniform(M.n, 1)
    As = A.to_scipy()
    x_ref, info_ref = fgmres(As, b, M.apply, restart=RESTART[name], rtol=1e-8)
    G = Gemslr.from_factors(A, part, M.factors())
    x, info = G.solve(torch.from_numpy(b).cuda(), restart=RESTART[name], rtol=1e-8)
    x = x.cpu().numpy()
    assert info[0]["converged"]
    assert abs(info[0]["iters"] - info_ref["iters"]) <= 1
    res = np.linalg.norm(b - As @ x) / np.linalg.norm(b)
    assert res <= 1e-8
    assert rel_err(x, x_ref) <= 1e-6


@pytest.mark.parametrize("name", ["c1", "small3d"])
def test_library_setup_matches_oracle_factors(torch_cuda, name):
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    G = Gemslr(A, part, **lib_opts(name))
    f = G.export_factors()
    ref = M.factors()
    for lf, rf in zip(f["levels"], ref["levels"]):
        for key in ("L", "U", "E", "F"):
            a, b = lf[key], rf[key]
            assert a.shape == b.shape and a.nnz == b.nnz, key
            assert np.array_equal(a.indices, b.indices) and np.array_equal(a.indptr, b.indptr), key
            assert np.allclose(a.data, b.data, rtol=1e-12, atol=0.0), key
        # low-rank terms agree as operators (basis-independent, Sec. 2.2)
        W, H = lf["W"], lf["H"]
        Wr, Hr = rf["W"], rf["H"]
        assert W.shape[1] == Wr.shape[1]
        s = W.shape[0]
        P = np.stack([gi.rhs_uniform(s, q) for q in range(3)], axis=1)
        C = W @ (H @ (W.T @ P))
        Cr = Wr @ (Hr @ (Wr.T @ P))
        assert rel_err(C, Cr) <= 5e-2
    for key in ("L", "U"):
        a, b = f["last"][key], ref["last"][key]
        assert np.array_equal(a.indices, b.indices) and np.allclose(a.data, b.data, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_library_setup_solves_to_tolerance(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    b = gi.rhs_uniform(A.n, 2)
    G = Gemslr(A, part, **lib_opts(name))
    x, info = G.solve(torch.from_numpy(b).cuda(), restart=RESTART[name], rtol=1e-8)
    x = x.cpu().numpy()
    assert info[0]["converged"] and info[0]["rel_res_true"] <= 1e-8
    res = np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b)
    assert res <= 1e-8
    st = G.stats()
    assert st["n"] == A.n and st["bytes_per_apply"] > 0
