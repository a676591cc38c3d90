"""GPU parity of the inner GMRES at the root level (Alg. 2 step 9).

With k inner steps, M^{-1} solves the root level's inexact Schur system
S_hat_0 y2 = z2 by k steps of right-preconditioned GMRES.  Both sides use the
same factors (exported by the oracle); the GPU orthogonalises with classical
Gram-Schmidt and a second pass, the oracle with modified Gram-Schmidt, so the
FP64 results agree to rounding: 1e-10 relative, like the standard
application.  The application is nonlinear; FGMRES must still match the
oracle's iteration count within one and reach the true residual tolerance.
"""
import ctypes

import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import fgmres
from tests.helpers import oracle_hierarchy, problem, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10
MIXED_TOL = 2e-2       # BF16 W and FP32 vectors, as for the standard application


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class _inner:
    """The cached oracle hierarchy with inner_steps set for the block."""

    def __init__(self, M, k):
        self.M, self.k = M, k

    def __enter__(self):
        self.old = self.M.inner_steps
        self.M.inner_steps = self.k
        return self.M

    def __exit__(self, *exc):
        self.M.inner_steps = self.old


@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("name", ["c1", "small3d", "shifted", "rank0", "tinyparts", "tiny2d"])
def test_inner_apply_matches_oracle(torch_cuda, name, k):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    G = Gemslr.from_factors(A, part, M.factors())
    G.set_inner_steps(k)
    with _inner(M, k):
        for seed in (41, 42):
            r = gi.rhs_uniform(M.n, seed)
            z_ref = M.apply(r)
            z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
            assert rel_err(z, z_ref) <= TOL, (name, k, rel_err(z, z_ref))
            assert np.max(np.abs(z - z_ref)) <= TOL * np.max(np.abs(z_ref))


def test_inner_apply_matches_oracle_c2(torch_cuda):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem("c2")
    M = oracle_hierarchy("c2")
    G = Gemslr.from_factors(A, part, M.factors())
    G.set_inner_steps(3)
    with _inner(M, 3):
        r = gi.rhs_uniform(M.n, 43)
        z_ref = M.apply(r)
    z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_err(z, z_ref) <= TOL


def test_inner_zero_rhs_and_switching_off(torch_cuda):
    """r = 0 gives z = 0 exactly (the beta = 0 path); steps = 0 restores the
    standard application bit for bit; the static entry point agrees."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr, _lib
    A, xyz, part = problem("small3d")
    M = oracle_hierarchy("small3d")
    G = Gemslr.from_factors(A, part, M.factors())
    r = torch.from_numpy(gi.rhs_uniform(M.n, 44)).cuda()
    z_std = G.apply(r)
    G.set_inner_steps(4)
    z0 = G.apply(torch.zeros_like(r)).cpu().numpy()
    assert np.all(z0 == 0.0)
    z_in = G.apply(r)
    lib = _lib.load()
    z_st = torch.full_like(r, float("nan"))
    st = lib.gemslr_apply_static(G._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z_st.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert torch.equal(z_st, z_in)
    assert not torch.equal(z_in, z_std)
    G.set_inner_steps(0)
    assert torch.equal(G.apply(r), z_std)
    for bad in (-1, 9):
        with pytest.raises(_lib.GemslrError):
            G.set_inner_steps(bad)


@pytest.mark.parametrize("name", ["c1", "small3d", "c2"])
def test_inner_mixed_apply_error_against_fp64_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    G = Gemslr.from_factors(A, part, M.factors(), precision="mixed")
    G.set_inner_steps(3)
    r = gi.rhs_uniform(M.n, 45)
    with _inner(M, 3):
        z_ref = M.apply(r)
    z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    err = rel_err(z, z_ref)
    assert 0.0 < err <= MIXED_TOL, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["shifted", "indef24"])
def test_fgmres_with_inner_matches_oracle(torch_cuda, name, precision):
    """Outer FGMRES with the inner steps: iterations within one of the
    oracle's (FP64; mixed within three), true residual <= 1e-8, and fewer
    iterations than the standard application on these shifted operators."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy(name)
    As = A.to_scipy()
    b = gi.rhs_uniform(M.n, 2)
    restart = 30
    with _inner(M, 3):
        _, ref = fgmres(As, b, M.apply, restart=restart, rtol=1e-8, maxit=600)
    assert ref["converged"]
    G = Gemslr.from_factors(A, part, M.factors(), precision=precision)
    bd = torch.from_numpy(b).cuda()
    _, std = G.solve(bd, restart=restart, rtol=1e-8, maxit=600)
    G.set_inner_steps(3)
    x, info = G.solve(bd, restart=restart, rtol=1e-8, maxit=600)
    res = np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b)
    assert info[0]["converged"] and res <= 1e-8
    slack = 1 if precision == "fp64" else 3
    assert abs(info[0]["iters"] - ref["iters"]) <= slack, (info[0]["iters"], ref["iters"])
    assert info[0]["iters"] < std[0]["iters"]
