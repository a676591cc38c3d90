"""Batched solve phase (many uneven systems, up to 8 right-hand sides each).

Each system is set up by the library exactly as a single system would be;
the batched M^{-1} (FP32 factors, BF16 W) must agree with the single-system
mixed-precision application of the same factors, and with the FP64 one to
the mixed-precision tolerance; every (system, rhs) FGMRES must reach 1e-8.
"""
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


def _systems(count, lo, hi, seed=3):
    from paper_2205_03224_gb300 import partition_geometric
    out = []
    for dims, beta in gi.batch_systems(count=count, seed=seed, lo=lo, hi=hi):
        A, xyz = gi.grid_operator(dims, beta=beta)
        out.append((A, partition_geometric(A, xyz, 3, 4)))
    return out


OPTS = dict(ilu="ilut", tau=1e-3, lfil=10, rank=6)


@pytest.fixture(scope="module")
def batch(torch_cuda):
    from paper_2205_03224_gb300 import GemslrBatch
    sy = _systems(7, 6, 13)
    B = GemslrBatch([a for a, _ in sy], [p for _, p in sy], **OPTS)
    return sy, B


def _stack(sy, nrhs, seed):
    cols = []
    for s, (A, _) in enumerate(sy):
        cols.append(np.stack([gi.rhs_uniform(A.n, seed + 100 * s + r) for r in range(nrhs)], axis=1).T.ravel())
    return np.concatenate(cols)


def test_batch_apply_matches_single_system(torch_cuda, batch):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    sy, B = batch
    nrhs = 3
    R = _stack(sy, nrhs, 5)
    Z = B.apply(torch.from_numpy(R).cuda(), nrhs).cpu().numpy()
    off = 0
    for A, part in sy:
        n = A.n
        Gm = Gemslr(A, part, precision="mixed", **OPTS)
        G64 = Gemslr(A, part, **OPTS)
        for r in range(nrhs):
            rv = R[off + r * n: off + (r + 1) * n]
            z = Z[off + r * n: off + (r + 1) * n]
            zm = Gm.apply(torch.from_numpy(rv).cuda()).cpu().numpy()
            z64 = G64.apply(torch.from_numpy(rv).cuda()).cpu().numpy()
            assert np.linalg.norm(z - zm) <= 1e-4 * np.linalg.norm(zm)
            assert np.linalg.norm(z - z64) <= 2e-2 * np.linalg.norm(z64)
        off += n * nrhs


@pytest.mark.parametrize("nrhs", [1, 8])
def test_batch_fgmres_converges_every_pair(torch_cuda, batch, nrhs):
    torch = torch_cuda
    sy, B = batch
    Bv = _stack(sy, nrhs, 9)
    X, info = B.solve(torch.from_numpy(Bv).cuda(), nrhs, restart=20, rtol=1e-8)
    X = X.cpu().numpy()
    off = 0
    for s, (A, _) in enumerate(sy):
        As = A.to_scipy()
        n = A.n
        for r in range(nrhs):
            b = Bv[off + r * n: off + (r + 1) * n]
            x = X[off + r * n: off + (r + 1) * n]
            res = np.linalg.norm(b - As @ x) / np.linalg.norm(b)
            assert res <= 1e-8, (s, r, res)
            assert info[s * nrhs + r]["converged"]
        off += n * nrhs
    st = B.stats()
    assert st["nsys"] == len(sy) and st["rows_couple"] in (64, 128, 256)
    rows0 = sum(int(p["level_ptr"][1]) for _, p in sy)          # the first level of every system
    assert st["lev0_rows"] == rows0 and st["lev0_l_bytes"] > 0 and st["lev0_u_bytes"] > 0


def test_batch_zero_rhs_and_single_system_iterations(torch_cuda, batch):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    sy, B = batch
    nrhs = 2
    Bv = _stack(sy, nrhs, 21)
    n0 = sy[0][0].n
    Bv[:n0] = 0.0                       # system 0, rhs 0 is zero
    X, info = B.solve(torch.from_numpy(Bv).cuda(), nrhs, restart=20, rtol=1e-8)
    X = X.cpu().numpy()
    assert np.all(X[:n0] == 0.0) and info[0]["converged"] and info[0]["iters"] == 0
    # the pairs iterate like the single-system mixed-precision solver
    A, part = sy[1]
    off = sum(a.n * nrhs for a, _ in sy[:1])
    b = Bv[off: off + A.n]
    Gm = Gemslr(A, part, precision="mixed", **OPTS)
    x, inf1 = Gm.solve(torch.from_numpy(b).cuda(), restart=20, rtol=1e-8)
    assert abs(inf1[0]["iters"] - info[1 * nrhs + 0]["iters"]) <= 2


def test_batch_host_loop_equals_graph(torch_cuda, batch, monkeypatch):
    """GEMSLR_SOLVE_GRAPH=0 drives the same kernels from the host (for
    profilers): the iterates are bit-identical to the graph's, with restarts."""
    torch = torch_cuda
    sy, B = batch
    nrhs = 4
    b = torch.from_numpy(_stack(sy, nrhs, 31)).cuda()
    Xg, ig = B.solve(b, nrhs, restart=1, rtol=1e-8)
    monkeypatch.setenv("GEMSLR_SOLVE_GRAPH", "0")
    Xh, ih = B.solve(b, nrhs, restart=1, rtol=1e-8)
    monkeypatch.delenv("GEMSLR_SOLVE_GRAPH")
    assert torch.equal(Xg, Xh)
    assert [(i["iters"], i["restarts"], i["converged"]) for i in ig] == \
        [(i["iters"], i["restarts"], i["converged"]) for i in ih]
    summary = [(i["iters"], i["restarts"]) for i in ig]
    assert max(i["restarts"] for i in ig) >= 1 and all(i["converged"] for i in ig), summary


def test_batch_splits_right_hand_sides_of_large_blocks(torch_cuda):
    """Blocks whose vector for 8 right-hand sides does not fit in shared
    memory are handled by several CTAs with fewer right-hand sides each; the
    result must still equal the single-system mixed application, for every
    right-hand side (each CTA of a block covers its own share)."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr, GemslrBatch, partition_geometric
    sy = []
    for dims, beta in [((30, 30, 28), 0.2), ((9, 8, 7), 0.1), ((24, 24, 24), 0.3)]:
        A, xyz = gi.grid_operator(dims, beta=beta)
        sy.append((A, partition_geometric(A, xyz, 3, 2)))
    B = GemslrBatch([a for a, _ in sy], [p for _, p in sy], **OPTS)
    assert B.stats()["rhs_per_cta"] in (1, 2, 4)
    nrhs = 8
    R = _stack(sy, nrhs, 17)
    Z = B.apply(torch.from_numpy(R).cuda(), nrhs).cpu().numpy()
    off = 0
    for A, part in sy:
        n = A.n
        Gm = Gemslr(A, part, precision="mixed", **OPTS)
        for r in range(nrhs):
            rv = R[off + r * n: off + (r + 1) * n]
            z = Z[off + r * n: off + (r + 1) * n]
            zm = Gm.apply(torch.from_numpy(rv).cuda()).cpu().numpy()
            assert np.linalg.norm(z - zm) <= 1e-4 * np.linalg.norm(zm), (n, r)
        off += n * nrhs


def test_batch_apply_matches_oracle(torch_cuda):
    """Every (system, rhs) of a small uneven batch against the FP64 oracle
    (Alg. 2), both sides on the oracle's factors with W rounded to BF16 (the
    batched path keeps W in BF16): what remains is FP32 rounding of the
    factors, vectors and sums, about 1e-6 relative, bounded at 1e-4."""
    torch = torch_cuda
    from oracle import OracleGemslr, multilevel_partition
    from paper_2205_03224_gb300 import GemslrBatch, partition_geometric
    from tests.helpers import rel_err, round_w_to_bf16
    sy, Ms, facs = [], [], []
    for dims, beta in gi.batch_systems(count=5, seed=13, lo=6, hi=12):
        A, xyz = gi.grid_operator(dims, beta=beta)
        As = A.to_scipy()
        part = partition_geometric(A, xyz, 3, 4)
        ref = multilevel_partition(As, xyz, 3, 4)
        assert np.array_equal(part["perm"], ref["perm"])
        M = OracleGemslr(As, ref, ilu="ilut", tau=1e-3, lfil=10, rank=6)
        facs.append(round_w_to_bf16(M))
        Ms.append(M)
        sy.append((A, part))
    B = GemslrBatch.from_factors([a for a, _ in sy], [p for _, p in sy], facs)
    for nrhs in (1, 8):
        R = _stack(sy, nrhs, 61)
        Z = B.apply(torch.from_numpy(R).cuda(), nrhs).cpu().numpy()
        off = 0
        for (A, _), M in zip(sy, Ms):
            n = A.n
            for r in range(nrhs):
                rv = R[off + r * n: off + (r + 1) * n]
                z = Z[off + r * n: off + (r + 1) * n]
                err = rel_err(z, M.apply(rv))
                assert 0.0 < err <= 1e-4, (n, r, err)
            off += n * nrhs
