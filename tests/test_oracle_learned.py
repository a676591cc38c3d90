"""Pins for the oracle of the learned interface correction (not in the paper):
the sparse 27-tap convolution against its dense matrix, backward against
central differences, the exact Schur complement of level l*, and the data
pairs (rho, S_hat^{-1} rho)."""
import numpy as np

import gemslr_inputs as gi
from oracle import OracleGemslr, multilevel_partition
from oracle.learned import (cnn, conv_backward, conv_forward, init_params, interface_stage, loss_and_grads,
                            net_forward, schur_dense, site_neighbors, training_pairs)


def _sites():
    # a 4x3x3 box with two holes
    c = np.array([(x, y, z) for z in range(3) for y in range(3) for x in range(4)])
    keep = np.ones(len(c), dtype=bool)
    keep[[5, 17]] = False
    return c[keep]


def test_neighbors_are_symmetric():
    nbr = site_neighbors(_sites())
    S = nbr.shape[0]
    for s in range(S):
        assert nbr[s, 13] == s
        for t in range(27):
            u = nbr[s, t]
            if u >= 0:
                assert nbr[u, 26 - t] == s


def test_conv_equals_dense_stencil_matrix():
    coords = _sites()
    nbr = site_neighbors(coords)
    S = len(coords)
    rng = np.random.default_rng(0)
    Cin, Cout = 2, 3
    W = rng.standard_normal((27, Cin, Cout))
    b = rng.standard_normal(Cout)
    x = rng.standard_normal((2, S, Cin))
    y = conv_forward(x, W, b, nbr)
    # dense: Y[:, :, co] = b + sum_ci A_{ci,co} X[:, :, ci], A built entry by entry from the offsets
    for co in range(Cout):
        acc = np.full((2, S), b[co])
        for ci in range(Cin):
            A = np.zeros((S, S))
            for s, c in enumerate(coords):
                for u, d in enumerate(coords):
                    off = d - c
                    if np.all(np.abs(off) <= 1):
                        t = (off[2] + 1) * 9 + (off[1] + 1) * 3 + (off[0] + 1)
                        A[s, u] = W[t, ci, co]
            acc += x[:, :, ci] @ A.T
        assert np.allclose(y[:, :, co], acc, rtol=1e-13, atol=1e-13)


def test_backward_matches_central_differences():
    coords = _sites()
    nbr = site_neighbors(coords)
    S = len(coords)
    params = init_params(channels=3, seed=5)
    rng = np.random.default_rng(1)
    rho = rng.standard_normal((2, S))
    tgt = rng.standard_normal((2, S))
    loss, grads = loss_and_grads(params, rho, tgt, nbr)
    h = 1e-6
    for l in range(4):
        W, b = params[l]
        for idx in [(0, 0, 0), (13, 0, W.shape[2] - 1), (26, W.shape[1] - 1, 0), (7, 0, 0)]:
            old = W[idx]
            W[idx] = old + h
            lp, _ = loss_and_grads(params, rho, tgt, nbr)
            W[idx] = old - h
            lm, _ = loss_and_grads(params, rho, tgt, nbr)
            W[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx)
        old = b[0]
        b[0] = old + h
        lp, _ = loss_and_grads(params, rho, tgt, nbr)
        b[0] = old - h
        lm, _ = loss_and_grads(params, rho, tgt, nbr)
        b[0] = old
        assert abs((lp - lm) / (2 * h) - grads[l][1][0]) <= 1e-6 * max(1.0, abs(grads[l][1][0]))
    # input gradient of one conv layer
    W = params[1][0]
    x = rng.standard_normal((1, S, 3))
    dy = rng.standard_normal((1, S, 3))
    dx, _, _ = conv_backward(x, W, nbr, dy)
    i = (0, 4, 1)
    xp = x.copy(); xp[i] += h
    xm = x.copy(); xm[i] -= h
    fd = (np.sum(dy * conv_forward(xp, W, np.zeros(3), nbr)) - np.sum(dy * conv_forward(xm, W, np.zeros(3), nbr))) / (2 * h)
    assert abs(fd - dx[i]) <= 1e-7 * max(1.0, abs(fd))


def test_relu_net_is_positively_homogeneous_without_bias():
    coords = _sites()
    nbr = site_neighbors(coords)
    params = init_params(channels=4, seed=2)
    x = np.random.default_rng(3).standard_normal((1, len(coords)))
    y1, _ = net_forward(params, x, nbr)
    y2, _ = net_forward(params, 3.0 * x, nbr)
    assert np.allclose(y2, 3.0 * y1, rtol=1e-12)


def test_schur_and_training_pairs():
    A, xyz = gi.grid_operator((9, 8, 7), beta=0.0, sigma=0.05)
    As = A.to_scipy()
    part = multilevel_partition(As, xyz, 3, 4)
    M = OracleGemslr(As, part, ilu="ilut", tau=1e-2, lfil=4, rank=4)
    l = 1
    S = schur_dense(M, l)
    lv = M.levels[l]
    # S y by the sparse route C y - E (LU)^-1 F y
    from oracle.ilu import lu_solve
    y = gi.rhs_uniform(S.shape[0], 4)
    e = lv["e"]
    sy = M.Ahat[e:, e:] @ y - lv["E"] @ lu_solve(lv["L"], lv["U"], lv["F"] @ y)
    assert np.allclose(S @ y, sy, rtol=1e-12, atol=1e-9 * np.abs(sy).max())
    R, T, S2 = training_pairs(M, l, 5, 77)
    assert np.allclose(S2 @ T.T, R.T, rtol=1e-9, atol=1e-9 * np.abs(R).max())
    # rho = z - S M_S^{-1} z for the method's own level-l application
    z = 2.0 * gi.uniform01(77, S.shape[0] * 5).reshape(5, -1)[0] - 1.0
    W, H = lv["W"], lv["H"]
    y2 = M.solve_level(z + W @ (H @ (W.T @ z)), l + 1)
    assert np.allclose(R[0], z - S @ y2, rtol=1e-10, atol=1e-10 * np.abs(R[0]).max())


def _two_level():
    A, xyz = gi.grid_operator((9, 8, 6), beta=0.3, sigma=0.05)
    As = A.to_scipy()
    part = multilevel_partition(As, xyz, 2, 4)
    M = OracleGemslr(As, part, ilu="ilut", tau=1e-2, lfil=3, rank=3)
    return As, xyz, part, M


def test_stage_with_ideal_network_solves_the_schur_system():
    """With net(x) = d S_hat^{-1} x the stage returns y2' = y2 + S_hat^{-1}(z2 - S_hat y2)
    = S_hat^{-1} z2 whatever y2 was.  With two levels (l* = 0 is the root) the
    application is then the exact inverse of A~ = [[LU, F], [E, C]], the matrix
    whose block elimination it performs (Sec. 2.3), for any incomplete factors.
    A wrong sign, a missing ||rho|| or a d applied the wrong way round breaks it."""
    As, xyz, part, M = _two_level()
    S = schur_dense(M, 0)
    d = float(np.mean(np.abs(np.diag(S))))
    M.stage = interface_stage(M, lambda x: d * np.linalg.solve(S, x))
    lv = M.levels[0]
    s, e = lv["s"], lv["e"]
    At = M.Ahat.toarray()
    LU = (np.eye(e - s) + lv["L"].toarray()) @ lv["U"].toarray()
    At[s:e, s:e] = LU
    r = gi.rhs_uniform(M.n, 8)
    z = M.apply_perm(r)
    assert np.allclose(z, np.linalg.solve(At, r), rtol=1e-9, atol=1e-9 * np.abs(z).max())
    M.stage = None
    assert not np.allclose(M.apply_perm(r), z, rtol=1e-3)     # the method alone is not exact here


def test_stage_with_zero_network_is_the_method():
    As, xyz, part, M = _two_level()
    r = gi.rhs_uniform(M.n, 9)
    z0 = M.apply_perm(r)
    M.stage = interface_stage(M, lambda x: np.zeros_like(x))
    assert np.array_equal(M.apply_perm(r), z0)


def test_stage_with_cnn_is_positively_homogeneous_and_changes_y():
    """N(rho) = (||rho||/d) net(rho/||rho||) is positively homogeneous even
    with biases, so the whole application stays homogeneous; the correction
    only touches the level's y2 and, through F, the y1 above it."""
    A, xyz = gi.grid_operator((9, 8, 7), beta=0.0, sigma=0.05)
    As = A.to_scipy()
    part = multilevel_partition(As, xyz, 3, 4)
    M = OracleGemslr(As, part, ilu="ilut", tau=1e-2, lfil=4, rank=4)
    e = M.levels[-1]["e"]
    nbr = site_neighbors(xyz[part["perm"][e:]])
    params = init_params(channels=4, seed=5)
    for l, (W, b) in enumerate(params):
        b[:] = 0.1 * (l + 1) * (1.0 - 2.0 * (np.arange(len(b)) % 2))
    r = gi.rhs_uniform(M.n, 10)
    z0 = M.apply_perm(r)
    M.stage = interface_stage(M, cnn(params, nbr))
    z1 = M.apply_perm(r)
    assert np.linalg.norm(z1 - z0) > 1e-3 * np.linalg.norm(z0)
    assert np.allclose(M.apply_perm(3.0 * r), 3.0 * z1, rtol=1e-12, atol=1e-12 * np.abs(z1).max())
    # rows of levels above l* change only through F y2: the first level's z1 part
    # differs, and the difference equals -(LU)^{-1} F (y2' - y2) of level 0's tail
    from oracle.ilu import lu_solve
    lv0 = M.levels[0]
    dy = z1[lv0["e"]:] - z0[lv0["e"]:]
    d1 = z1[:lv0["e"]] - z0[:lv0["e"]]
    assert np.allclose(d1, -lu_solve(lv0["L"], lv0["U"], lv0["F"] @ dy), rtol=1e-9,
                       atol=1e-9 * np.abs(d1).max())
