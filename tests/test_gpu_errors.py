"""Argument errors at the C ABI: each returns GEMSLR_ERR_ARG with a message
and leaves the library usable (a valid call afterwards succeeds)."""
import ctypes

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


def _setup_status(A, part):
    from paper_2205_03224_gb300 import Gemslr, _lib
    try:
        Gemslr(A, part, ilu="ilu0", rank=2)
    except _lib.GemslrError as e:
        return e.status, str(e)
    return 0, ""


def test_invalid_matrices_are_rejected(torch_cuda):
    from paper_2205_03224_gb300 import partition_geometric
    A, xyz = gi.grid_operator((6, 5))
    part = partition_geometric(A, xyz, 2, 2)
    n = A.n
    bad_col = gi.CSR(n, A.rowptr.copy(), A.colind.copy(), A.val.copy())
    bad_col.colind[5] = n                                   # column out of range
    unsorted = gi.CSR(n, A.rowptr.copy(), A.colind.copy(), A.val.copy())
    p0 = unsorted.rowptr[7]
    unsorted.colind[p0], unsorted.colind[p0 + 1] = unsorted.colind[p0 + 1], unsorted.colind[p0]
    empty = gi.CSR(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    for M, word in ((bad_col, "out of range"), (unsorted, "ascending"), (empty, "without entries")):
        st, msg = _setup_status(M, part)
        assert st == 1 and word in msg, (st, msg)
    st, _ = _setup_status(A, part)                         # still usable
    assert st == 0


def test_invalid_solve_options_are_rejected(torch_cuda):
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr, _lib, partition_geometric
    A, xyz = gi.grid_operator((8, 7))
    G = Gemslr(A, partition_geometric(A, xyz, 2, 2), ilu="ilu0", rank=2)
    lib = _lib.load()
    b = torch.from_numpy(gi.rhs_uniform(A.n, 1)).cuda()
    x = torch.empty_like(b)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for opts in (_lib.SolveOpts(0, 10, 1e-8, 0), _lib.SolveOpts(10, 0, 1e-8, 0), _lib.SolveOpts(10, 10, 0.0, 0),
                 _lib.SolveOpts(10, 10, 1e-8, 2), _lib.SolveOpts(400, 10, 1e-8, 0)):
        info = (_lib.SolveInfo * 1)()
        st = lib.gemslr_fgmres_solve(G._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1,
                                     ctypes.byref(opts), info, stream)
        assert st == 1, (opts.restart, opts.maxit, opts.rtol, opts.ortho)
        assert lib.gemslr_last_error().decode()
    xs, info = G.solve(b, restart=20, rtol=1e-8)            # still usable
    assert info[0]["converged"]


def test_factor_file_round_trip_and_corruption(torch_cuda, tmp_path):
    """gemslr_save_factors / gemslr_load_factors: the reloaded handle applies the
    same M^{-1} bit for bit (mixed precision too); a truncated file, a foreign
    file and a file for another matrix size are rejected with ERR_ARG."""
    torch = torch_cuda
    from paper_2205_03224_gb300 import Gemslr, _lib, partition_geometric
    A, xyz = gi.grid_operator((13, 11, 9), beta=0.4)
    part = partition_geometric(A, xyz, 3, 8)
    G = Gemslr(A, part, ilu="ilut", tau=1e-2, lfil=5, rank=5, precision="mixed")
    path = tmp_path / "factors.bin"
    G.save_factors(str(path))
    G2 = Gemslr.load_factors(A, part, str(path), precision="mixed")
    r = torch.from_numpy(gi.rhs_uniform(A.n, 5)).cuda()
    assert torch.equal(G.apply(r), G2.apply(r))
    data = path.read_bytes()
    bad = tmp_path / "truncated.bin"
    bad.write_bytes(data[: len(data) // 2])
    foreign = tmp_path / "foreign.bin"
    foreign.write_bytes(b"NOTGEMSL" + data[8:])
    A2, xyz2 = gi.grid_operator((12, 11, 9), beta=0.4)
    part2 = partition_geometric(A2, xyz2, 3, 8)
    for (M, P, f) in ((A, part, bad), (A, part, foreign), (A2, part2, path), (A, part, tmp_path / "missing.bin")):
        with pytest.raises(_lib.GemslrError) as e:
            Gemslr.load_factors(M, P, str(f), precision="mixed")
        assert e.value.status == 1
