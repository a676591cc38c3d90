"""Learned interface correction (an addition to the paper's method).

The GPU network (BF16 weights, FP32 accumulation) must reproduce the FP64
oracle's loss and gradients at the same (BF16-rounded) weights; training
must reduce the loss; with the stage on, FGMRES must still reach 1e-8, in
fewer iterations than without it."""
import numpy as np
import pytest

import gemslr_inputs as gi
from oracle.learned import init_params, loss_and_grads, site_neighbors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bf16(a):
    """Round float64 -> float32 -> bfloat16 (nearest even) -> float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def _unflat(vec, C):
    dims = [1, C, C, C, 1]
    out, off = [], 0
    for l in range(4):
        nw = 27 * dims[l] * dims[l + 1]
        W = vec[off:off + nw].reshape(27, dims[l], dims[l + 1])
        b = vec[off + nw: off + nw + dims[l + 1]]
        out.append([W.copy(), b.copy()])
        off += nw + dims[l + 1]
    return out


@pytest.fixture(scope="module")
def handle(torch_cuda):
    from paper_2205_03224_gb300 import Gemslr, partition_geometric
    A, xyz = gi.stencil3d(14, sigma=0.05)
    part = partition_geometric(A, xyz, 3, 8)
    G = Gemslr(A, part, ilu="ilut", tau=1e-3, lfil=10, rank=6)
    return A, xyz, part, G


def test_gradients_match_oracle(handle):
    A, xyz, part, G = handle
    C = 8
    G.learned_train(xyz, channels=C, npairs=64, epochs=0, batch=16, seed=7)
    info = G.learned_info()
    S = info["sites"]
    # same seeded initialisation on both sides
    ref = init_params(channels=C, seed=7)
    assert np.allclose(G.learned_params(), _flat(ref), rtol=1e-6, atol=1e-7)
    # sites = the deepest level's unknowns in the multilevel order
    e = int(part["level_ptr"][-2])
    nbr = site_neighbors(xyz[part["perm"][e:]])
    assert nbr.shape[0] == S
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, S))
    y = rng.standard_normal((5, S))
    loss, grad = G.learned_loss_grad(x, y)
    pr = [[_bf16(W), b.copy()] for W, b in ref]   # the GPU passes use BF16 copies of the weights
    xr, yr = np.asarray(x, np.float32).astype(np.float64), np.asarray(y, np.float32).astype(np.float64)
    lref, gref = loss_and_grads(pr, xr, yr, nbr)
    gflat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in gref])
    assert abs(loss - lref) <= 1e-4 * abs(lref)
    assert np.linalg.norm(grad - gflat) <= 1e-3 * np.linalg.norm(gflat)


def test_training_reduces_loss_and_solve_converges(torch_cuda, handle):
    torch = torch_cuda
    A, xyz, part, G = handle
    b = torch.from_numpy(gi.rhs_uniform(A.n, 4)).cuda()
    G.learned_enable(False) if _has_stage(G) else None
    x0, i0 = G.solve(b, restart=40, rtol=1e-8)
    hist = G.learned_train(xyz, channels=16, npairs=2048, epochs=6, batch=32, lr=2e-3, seed=4)
    assert hist[-1] < hist[0]
    x1, i1 = G.solve(b, restart=40, rtol=1e-8)
    res = np.linalg.norm(gi.rhs_uniform(A.n, 4) - A.to_scipy() @ x1.cpu().numpy()) / np.linalg.norm(b.cpu().numpy())
    assert i1[0]["converged"] and res <= 1e-8
    # what the network gains: on this shifted operator the trained stage cuts the
    # outer iterations at the same accuracy (measured 21 -> 13 on the GB300)
    assert i1[0]["iters"] <= i0[0]["iters"] - 3, (i0[0]["iters"], i1[0]["iters"])
    G.learned_enable(False)
    x2, i2 = G.solve(b, restart=40, rtol=1e-8)
    assert i2[0]["iters"] == i0[0]["iters"]        # switching the stage off restores the method


def _has_stage(G):
    try:
        G.learned_info()
        return True
    except Exception:
        return False


def test_in_apply_stage_matches_oracle(torch_cuda):
    """One M^{-1} application with the stage on, element by element against
    the oracle's restatement: rho = z2 - S_hat y2 at l* = nlev - 2,
    y2 += (||rho|| / d) net(rho / ||rho||), then the back-substitution with F.
    Both sides use the oracle's factors and the same network (weights rounded
    to BF16, biases to FP32, as the GPU keeps them).  The stage's own
    contribution (application with it minus without it) must agree to FP32
    accuracy, which a wrong sign, scale, level or site order would break."""
    torch = torch_cuda
    from oracle import OracleGemslr, multilevel_partition
    from oracle.learned import cnn, interface_stage, schur_dense
    from paper_2205_03224_gb300 import Gemslr, partition_geometric
    A, xyz = gi.grid_operator((12, 11, 10), beta=0.0, sigma=0.05)
    As = A.to_scipy()
    part = partition_geometric(A, xyz, 3, 8)
    ref_part = multilevel_partition(As, xyz, 3, 8)
    assert np.array_equal(part["perm"], ref_part["perm"])
    M = OracleGemslr(As, ref_part, ilu="ilut", tau=1e-3, lfil=10, rank=5)
    G = Gemslr.from_factors(A, part, M.factors())
    C = 8
    G.learned_train(xyz, channels=C, npairs=16, epochs=0, batch=16, seed=3)
    params = init_params(channels=C, seed=11)
    for l, (W, b) in enumerate(params):
        b[:] = 0.05 * (l + 1) * (1.0 - 2.0 * (np.arange(len(b)) % 2))
    G.learned_params(_flat(params))
    pr = [[_bf16(W), np.asarray(b, np.float32).astype(np.float64)] for W, b in params]
    lstar = M.nlev - 2
    e = M.levels[lstar]["e"]
    nbr = site_neighbors(xyz[part["perm"][e:]])
    d = float(np.mean(np.abs(np.diag(schur_dense(M, lstar)))))
    info = G.learned_info()
    assert info["sites"] == nbr.shape[0]
    assert abs(info["dscale"] - d) <= 1e-12 * d
    for seed in (41, 42):
        r = gi.rhs_uniform(A.n, seed)
        rd = torch.from_numpy(r).cuda()
        G.learned_enable(True)
        z_on = G.apply(rd).cpu().numpy()
        G.learned_enable(False)
        z_off = G.apply(rd).cpu().numpy()
        M.stage = None
        z0 = M.apply(r)
        M.stage = interface_stage(M, cnn(pr, nbr), d)
        z1 = M.apply(r)
        M.stage = None
        assert np.linalg.norm(z_off - z0) <= 1e-10 * np.linalg.norm(z0)
        delta, delta_ref = z_on - z_off, z1 - z0
        assert np.linalg.norm(delta_ref) >= 1e-3 * np.linalg.norm(z0)
        assert np.linalg.norm(delta - delta_ref) <= 1e-4 * np.linalg.norm(delta_ref), seed
        assert np.linalg.norm(z_on - z1) <= 1e-4 * np.linalg.norm(z1)
