"""Pins for the shared synthetic-input generators."""
import os

import numpy as np

import gemslr_inputs as gi

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLD, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, *outs = [int(t) for t in line.split()]
        got = gi.splitmix64(seed, 3)
        assert [int(v) for v in got] == outs


def test_rhs_range_and_determinism():
    b = gi.rhs_uniform(10000, 7)
    assert b.min() >= -1.0 and b.max() < 1.0
    assert abs(b.mean()) < 0.05
    assert np.array_equal(b, gi.rhs_uniform(10000, 7))
    assert not np.array_equal(b, gi.rhs_uniform(10000, 8))


def test_laplacian_closed_forms():
    A, xyz = gi.laplace2d(32)
    assert A.n == 1024 and A.nnz == 5 * 1024 - 4 * 32
    D = A.to_dense()
    h2 = (1.0 / 33) ** -2
    assert np.allclose(np.diag(D), 4 * h2)
    assert np.allclose(D, D.T)
    # interior rows sum to zero, rows touching one boundary side sum to h^-2
    s = D.sum(axis=1).reshape(32, 32)
    assert np.allclose(s[1:-1, 1:-1], 0.0)
    assert np.allclose(s[0, 1:-1], h2)
    # eigenvalues of the 1-D second difference: lam_jk = h^-2 (4 - 2cos(j pi h) - 2cos(k pi h))
    ev = np.sort(np.linalg.eigvalsh(D))
    j = np.arange(1, 33)
    lam1 = 2 - 2 * np.cos(j * np.pi / 33)
    ref = np.sort((lam1[:, None] + lam1[None, :]).ravel()) * h2
    assert np.allclose(ev, ref, rtol=1e-10)


def test_convection_diffusion_stencil():
    N, beta = 6, 0.7
    A, xyz = gi.stencil3d(N, beta=beta)
    D = A.to_dense()
    h = 1.0 / (N + 1)
    assert A.nnz == 7 * N**3 - 6 * N**2
    i = 1 + N * 2 + N * N * 3                    # interior point (1,2,3)
    assert np.isclose(D[i, i], 6 / h**2)
    for stride in (1, N, N * N):
        assert np.isclose(D[i, i + stride], -1 / h**2 + beta / (2 * h))
        assert np.isclose(D[i, i - stride], -1 / h**2 - beta / (2 * h))
    # skew part is the centred convection term only
    K = 0.5 * (D - D.T)
    assert np.isclose(np.abs(K).max(), beta / (2 * h))


def test_shift_and_batch_sampler():
    N = 5
    A0, _ = gi.stencil3d(N)
    A1, _ = gi.stencil3d(N, sigma=0.05)
    h = 1.0 / (N + 1)
    assert np.allclose(A0.to_dense() - A1.to_dense(), 0.05 / h**2 * np.eye(N**3))
    sy = gi.batch_systems()
    assert len(sy) == 96
    for dims, beta in sy:
        assert all(16 <= d <= 48 for d in dims) and 0.0 <= beta < 0.5
    assert sy == gi.batch_systems()
