"""Full-size parity of M^{-1} (Alg. 2) on the indefinite 128^3 (mixed
precision) and 96^3 (learned-stage) workloads, in the launch configuration of
`bench.py`: the library sets the hierarchy up, exports its FP64 factors, and
the oracle applies Alg. 2 with exactly those factors (OracleGemslr.from_factors,
nothing refactored).  The FP64 kernels on the same factors agree with the
oracle to 1e-10 (measured: 4e-16); the mixed kernels (FP32 factors and vectors, BF16 W) agree
with the oracle fed the BF16-rounded W up to FP32 rounding.
"""
import functools

import numpy as np
import pytest

import gemslr_inputs as gi
from oracle import OracleGemslr
from tests.helpers import bf16, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@functools.lru_cache(maxsize=None)
def _library_setup(name):
    """(A, partition, exported FP64 factors) of the library's own set-up of a config."""
    from paper_2205_03224_gb300 import Gemslr, partition_geometric
    c = gi.CONFIGS[name]
    A, xyz, _ = gi.config_problem(name)
    part = partition_geometric(A, xyz, c["nlev"], c["p"], local_from=c.get("local_from"))
    G = Gemslr(A, part, ilu=c["ilu"], tau=c["tau"], lfil=c["lfil"], rank=c["rank"], precision="mixed")
    fac = G.export_factors()
    G.close()
    return A, part, fac


def _with_bf16_w(fac):
    out = dict(levels=[dict(lv) for lv in fac["levels"]], last=fac["last"])
    for lv in out["levels"]:
        lv["W"] = bf16(lv["W"])
    return out


@pytest.mark.parametrize("name", ["c3", "c5"])
def test_full_size_fp64_apply_matches_oracle_on_library_factors(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, part, fac = _library_setup(name)
    M = OracleGemslr.from_factors(A.to_scipy(), part, fac)
    G = Gemslr.from_factors(A, part, fac)
    for seed in (21, 22):
        r = gi.rhs_uniform(A.n, seed)
        z_ref = M.apply(r)
        z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel_err(z, z_ref) <= 1e-10, name
        assert np.max(np.abs(z - z_ref)) <= 1e-10 * np.max(np.abs(z_ref))
    G.close()


def test_full_size_mixed_apply_matches_oracle_with_bf16_w(torch_cuda):
    """The 128^3 mixed-precision application (the c3 bench line's M^-1) against
    the oracle fed the same factors with W rounded to BF16: what remains is FP32
    rounding of factors, vectors and sums, amplified by the indefinite
    operator's levels."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr
    A, part, fac = _library_setup("c3")
    M = OracleGemslr.from_factors(A.to_scipy(), part, _with_bf16_w(fac))
    G = Gemslr.from_factors(A, part, fac, precision="mixed")
    r = gi.rhs_uniform(A.n, 23)
    z_ref = M.apply(r)
    z = G.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    err = rel_err(z, z_ref)
    assert 0.0 < err <= 1e-5, err          # measured on the GB300: 6.8e-8
    G.close()


def test_full_size_batched_apply_matches_oracle(torch_cuda):
    """The batched workload at full size (96 uneven convection-diffusion systems,
    sides 16..48, 8 right-hand sides each, the c4 bench line's launch
    configuration): every system's hierarchy from the library's own set-up,
    batched through gemslr_setup_batch_from_factors, against the oracle on the
    same factors with W rounded to BF16, for the first and the last
    right-hand side of every system (FP32 rounding only)."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr, GemslrBatch, partition_geometric
    c = gi.CONFIGS["c4"]
    As, parts, facs, Ms = [], [], [], []
    for dims, beta in gi.batch_systems(count=c["count"], seed=c["seed"]):
        A, xyz = gi.grid_operator(dims, beta=beta)
        part = partition_geometric(A, xyz, c["nlev"], c["p"])
        G = Gemslr(A, part, ilu=c["ilu"], tau=c["tau"], lfil=c["lfil"], rank=c["rank"])
        fac = G.export_factors()
        G.close()
        As.append(A)
        parts.append(part)
        facs.append(fac)
        Ms.append(OracleGemslr.from_factors(A.to_scipy(), part, _with_bf16_w(fac)))
    B = GemslrBatch.from_factors(As, parts, facs)
    nrhs = c["nrhs"]
    R = np.concatenate([np.stack([gi.rhs_uniform(A.n, 7000 + 10 * s + r) for r in range(nrhs)], axis=1).T.ravel()
                        for s, A in enumerate(As)])
    Z = B.apply(torch.from_numpy(R).cuda(), nrhs).cpu().numpy()
    off = 0
    for A, M in zip(As, Ms):
        n = A.n
        for r in (0, nrhs - 1):
            rv = R[off + r * n: off + (r + 1) * n]
            err = rel_err(Z[off + r * n: off + (r + 1) * n], M.apply(rv))
            assert 0.0 < err <= 1e-4, (n, r, err)
        off += n * nrhs
    assert off == R.size
    B.close()
