"""GPU parity of the complex-shifted method (Sec. 5.2.3) against the oracle.

The diagonal blocks are factored as B + i alpha I (alpha = shift * sum |a_ii| / n),
the corrections W H W^H come from the Arnoldi in complex arithmetic and
M^{-1} and FGMRES run in complex FP64.  The application is compared with the
oracle on the oracle's own factors (imported through the C ABI), the library's
set-up with the oracle's factors, and the complex FGMRES with the oracle's
complex FGMRES.
"""
import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import fgmres
from tests.helpers import lib_opts, oracle_hierarchy_z, problem, rel_err, rhs_complex

pytestmark = pytest.mark.gpu
TOL = 1e-10
SHIFT = 0.05


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _lib_from_oracle(name, shift=SHIFT):
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy_z(name, shift)
    return Gemslr.from_factors(A, part, M.factors()), M


# c2local: the full 64^3 workload of `bench.py --workload c2z`, in its launch configuration
@pytest.mark.parametrize("name", ["c1", "small3d", "shifted", "tinyparts", "bigblock", "indef24", "c2local"])
def test_complex_apply_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    G, M = _lib_from_oracle(name)
    assert G.complex and M.alpha > 0
    assert any(np.iscomplexobj(lv["W"]) and lv["W"].shape[1] > 0 for lv in M.levels) or name == "tinyparts"
    for seed in (11, 12):
        r = rhs_complex(M.n, seed)
        z_ref = M.apply(r)
        z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel_err(z, z_ref) <= TOL, name
        assert np.max(np.abs(z - z_ref)) <= TOL * np.max(np.abs(z_ref))
    r = gi.rhs_uniform(M.n, 13)                         # a real right-hand side
    z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_err(z, M.apply(r)) <= TOL


def test_complex_apply_multi_rhs_zero_and_refusals(torch_cuda):
    torch = torch_cuda
    from paper_2205_03224_gb300 import _lib as L
    import ctypes
    G, M = _lib_from_oracle("small3d")
    R = np.stack([rhs_complex(M.n, s) for s in (1, 2, 3)], axis=1)
    Z = G.apply(torch.from_numpy(R).cuda()).cpu().numpy()
    for c in range(3):
        assert rel_err(Z[:, c], M.apply(R[:, c])) <= TOL
    z0 = G.apply(torch.zeros(M.n, dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert np.all(z0 == 0.0)
    lib = L.load()
    r = torch.from_numpy(gi.rhs_uniform(M.n, 1)).cuda()
    z = torch.empty_like(r)
    st = lib.gemslr_apply(G._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), 1, None)
    assert L.STATUS[st] == "ERR_ARG"            # the real entry point refuses a complex handle
    assert "complex" in lib.gemslr_last_error().decode()


@pytest.mark.parametrize("name", ["c1", "small3d", "shifted"])
def test_complex_library_setup_matches_oracle_factors(torch_cuda, name):
    """The library's complex ILU of B + i alpha I equals the oracle's entrywise;
    its complex Krylov-Schur correction agrees as an operator (W H W^H does not
    depend on the basis of the wanted invariant subspace)."""
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem(name)
    M = oracle_hierarchy_z(name, SHIFT)
    G = Gemslr(A, part, shift=SHIFT, **lib_opts(name))
    assert G.complex
    f = G.export_factors()
    ref = M.factors()
    for lf, rf in zip(f["levels"], ref["levels"]):
        for key in ("L", "U", "E", "F"):
            a, b = lf[key], rf[key]
            assert a.shape == b.shape and a.nnz == b.nnz, key
            assert np.array_equal(a.indices, b.indices) and np.array_equal(a.indptr, b.indptr), key
            assert np.allclose(a.data, b.data, rtol=1e-12, atol=0.0), key
        W, H = lf["W"], lf["H"]
        Wr, Hr = rf["W"], rf["H"]
        assert W.shape[1] == Wr.shape[1]
        s = W.shape[0]
        P = np.stack([rhs_complex(s, q) for q in range(3)], axis=1)
        C = W @ (H @ (W.conj().T @ P))
        Cr = Wr @ (Hr @ (Wr.conj().T @ P))
        assert rel_err(C, Cr) <= 5e-2
    for key in ("L", "U"):
        a, b = f["last"][key], ref["last"][key]
        assert np.array_equal(a.indices, b.indices) and np.allclose(a.data, b.data, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name", ["c1", "small3d", "shifted", "indef24", "c2local"])
def test_complex_fgmres_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    A, xyz, part = problem(name)
    G, M = _lib_from_oracle(name)
    As = A.to_scipy()
    b = gi.rhs_uniform(M.n, 1)
    restart = 50 if name == "c2local" else 30
    x_ref, info_ref = fgmres(As, b, M.apply, restart=restart, rtol=1e-8, cplx=True)
    assert info_ref["converged"]
    x, info = G.solve(torch.from_numpy(b).cuda(), restart=restart, rtol=1e-8)
    x = x.cpu().numpy()
    assert np.iscomplexobj(x)
    assert info[0]["converged"]
    assert abs(info[0]["iters"] - info_ref["iters"]) <= 1, (info[0]["iters"], info_ref["iters"])
    res = np.linalg.norm(b - As @ x) / np.linalg.norm(b)
    assert res <= 1e-8
    assert rel_err(x, x_ref) <= 1e-6


def test_complex_fgmres_residual_history_matches_oracle(torch_cuda):
    """Within one cycle the Givens estimate after k steps equals the oracle's
    (FGMRES minimises the same residual over the same space) and the true
    residual of the returned iterate."""
    torch = torch_cuda
    A, xyz, part = problem("indef24")
    G, M = _lib_from_oracle("indef24")
    As = A.to_scipy()
    b = rhs_complex(M.n, 2)
    _, info_ref = fgmres(As, b, M.apply, restart=40, rtol=1e-14, maxit=20, cplx=True)
    hist = info_ref["hist"]
    assert len(hist) == 20
    bd = torch.from_numpy(b).cuda()
    for k in (1, 2, 5, 9, 14, 20):
        x, info = G.solve(bd, restart=40, rtol=1e-14, maxit=k, check=False)
        est = info[0]["rel_res_est"]
        true = np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b)
        assert info[0]["iters"] == k
        assert abs(est - hist[k - 1]) <= 1e-6 * hist[k - 1], (k, est, hist[k - 1])
        assert abs(true - est) <= 1e-6 * est, (k, est, true)


def test_complex_library_setup_solves_indefinite(torch_cuda):
    """The library's complex set-up on the indefinite 24^3 operator (shift
    0.1 h^-2) solves to 1e-8 within one iteration of the oracle's count."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, xyz, part = problem("indef24")
    M = oracle_hierarchy_z("indef24", SHIFT)
    As = A.to_scipy()
    b = gi.rhs_uniform(A.n, 3)
    _, info_ref = fgmres(As, b, M.apply, restart=30, rtol=1e-8, cplx=True)
    G = Gemslr(A, part, shift=SHIFT, **lib_opts("indef24"))
    x, info = G.solve(torch.from_numpy(b).cuda(), restart=30, rtol=1e-8)
    x = x.cpu().numpy()
    assert info[0]["converged"]
    assert abs(info[0]["iters"] - info_ref["iters"]) <= 1, (info[0]["iters"], info_ref["iters"])
    assert np.linalg.norm(b - As @ x) / np.linalg.norm(b) <= 1e-8
    st = G.stats()
    assert st["bytes_per_apply"] > 0 and st["levels"][0]["wavefronts_L"] > 0


def test_complex_option_combinations_are_refused(torch_cuda):
    from paper_2205_03224_gb300 import Gemslr, GemslrBatch
    from paper_2205_03224_gb300._lib import GemslrError
    A, xyz, part = problem("c1")
    for extra in (dict(precision="mixed"), dict(ilu="ilu0_device"), dict(lowrank="randomized")):
        with pytest.raises(GemslrError, match="ERR_UNSUPPORTED"):
            Gemslr(A, part, shift=SHIFT, rank=4, **extra)
    with pytest.raises(GemslrError, match="ERR_UNSUPPORTED"):
        GemslrBatch([A], [part], shift=SHIFT, rank=4)
    G = Gemslr(A, part, shift=SHIFT, rank=4)
    with pytest.raises(GemslrError, match="ERR_UNSUPPORTED"):
        G.save_factors("/tmp/never_written.gemslr")
    with pytest.raises(GemslrError, match="ERR_ARG"):
        G.set_inner_steps(2)
