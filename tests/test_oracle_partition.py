"""Pins for the oracle's multilevel reordering (Alg. 3, Sec. 3)."""
import os

import numpy as np
import scipy.sparse as sp

import gemslr_inputs as gi
from oracle.partition import (check_partition, level_blocks, multilevel_partition,
                              rcm_order, separator, rcb_parts)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold_c1():
    d = {}
    for line in open(os.path.join(GOLD, "c1_partition.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = [int(t) for t in v]
    return d


def test_c1_sizes_match_hand_derivation():
    A, xyz = gi.laplace2d(32)
    P = multilevel_partition(A.to_scipy(), xyz, 2, 4)
    g = _gold_c1()
    s, e, bp = level_blocks(P, 0)
    assert list(np.diff(bp)) == g["blocks"]
    assert P["level_ptr"][2] - P["level_ptr"][1] == g["separator"][0]
    check_partition(A.to_scipy(), P)


def test_vertex_separator_validity_brute_force():
    # T9: disjoint parts, union is V, no edge joins two different interiors
    for dims, nlev, p in [((9, 7, 6), 3, 4), ((12, 11), 3, 8), ((10, 10, 10), 4, 8)]:
        A, xyz = gi.grid_operator(dims, beta=0.3)
        As = A.to_scipy()
        P = multilevel_partition(As, xyz, nlev, p)
        check_partition(As, P)
        # brute force on the dense pattern, level by level
        D = (As.toarray() != 0)
        perm = P["perm"]
        for l in range(nlev - 1):
            s, e, bp = level_blocks(P, l)
            for a in range(len(bp) - 1):
                for b in range(len(bp) - 1):
                    if a == b:
                        continue
                    ia = perm[bp[a]:bp[a + 1]]
                    ib = perm[bp[b]:bp[b + 1]]
                    assert not D[np.ix_(ia, ib)].any()


def test_separator_rule_on_a_path():
    # path 0-1-2-3-4-5 split in two parts {0,1,2} {3,4,5}: only 3 is a separator
    n = 6
    G = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    verts = np.arange(n)
    part = np.array([0, 0, 0, 1, 1, 1])
    assert list(np.flatnonzero(separator(verts, part, G))) == [3]


def test_rcb_median_split():
    xyz = np.zeros((16, 3), dtype=np.int32)
    xyz[:, 0] = np.arange(16) % 4
    xyz[:, 1] = np.arange(16) // 4
    part = rcb_parts(np.arange(16), xyz, 4)
    # x-extent == y-extent -> first split on x, then on y in each half
    assert list(part.reshape(4, 4)[0]) == [0, 0, 2, 2]
    assert list(part.reshape(4, 4)[3]) == [1, 1, 3, 3]


def test_rcm_on_path_and_grid():
    n = 7
    G = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    # start: min degree, lowest index -> 0; BFS gives 0..6; reversed
    assert list(rcm_order(G)) == list(range(n - 1, -1, -1))
    # shuffled path: RCM recovers a banded (bandwidth 1) ordering
    rng = np.random.default_rng(0)
    q = rng.permutation(n)
    Gq = G[q][:, q]
    o = rcm_order(Gq)
    Go = Gq[o][:, o].tocoo()
    assert np.abs(Go.row - Go.col).max() == 1
    assert sorted(o.tolist()) == list(range(n))
    # 2-D grid: RCM bandwidth is no larger than the natural lexicographic one
    A, _ = gi.laplace2d(9)
    S = A.to_scipy()
    S.setdiag(0)
    S.eliminate_zeros()
    o = rcm_order(S)
    So = S[o][:, o].tocoo()
    assert np.abs(So.row - So.col).max() <= 9


def test_c2_level_sizes():
    A, xyz = gi.stencil3d(64, beta=0.1)
    P = multilevel_partition(A.to_scipy(), xyz, 4, 64)
    sizes = np.diff(P["level_ptr"])
    # 64 interior cubes 15^3..16^3; separators 35,163 -> 4,093 -> 852
    assert sizes[0] == 262144 - 35163
    assert sizes[1] + sizes[2] + sizes[3] == 35163
    assert sizes[2] + sizes[3] == 4093
    assert sizes[3] == 852
    s, e, bp = level_blocks(P, 0)
    d = np.diff(bp)
    assert d.min() == 15**3 and d.max() == 16**3


def test_local_order_keeps_blocks_and_separates_neighbours():
    """The local order (Sec. 3.2) only permutes inside the blocks of the chosen
    levels; inside a block the colour key never decreases and equal keys keep
    their original order; two vertices of one class are never neighbours in
    the stencil graph (brute force), so each class is an independent set."""
    from oracle.partition import level_blocks, local_order
    A, xyz = gi.grid_operator((11, 9, 7), beta=0.3)
    As = A.to_scipy()
    part = multilevel_partition(As, xyz, 4, 8)
    loc = local_order(part, xyz, 1)
    check_partition(As, loc)
    G = (abs(As) + abs(As.T)).tocsr()
    c = np.asarray(xyz, dtype=np.int64)
    key = 8 * (((c[:, 0] // 2) % 2) + 2 * ((c[:, 1] // 2) % 2) + 4 * ((c[:, 2] // 2) % 2)) + \
        (c[:, 0] % 2) + 2 * (c[:, 1] % 2) + 4 * (c[:, 2] % 2)
    for l in range(4):
        _, _, bp = level_blocks(part, l)
        for j in range(len(bp) - 1):
            a, b = bp[j], bp[j + 1]
            old, new = part["perm"][a:b], loc["perm"][a:b]
            assert sorted(old) == sorted(new)
            if l == 0:
                assert np.array_equal(old, new)            # level 0 untouched
                continue
            k = key[new]
            assert np.all(np.diff(k) >= 0)
            pos = {v: i for i, v in enumerate(old)}
            for cls in np.unique(k):
                members = new[k == cls]
                assert all(pos[members[i]] < pos[members[i + 1]] for i in range(len(members) - 1))
                ms = set(members.tolist())
                for v in members:
                    nb = G.indices[G.indptr[v]:G.indptr[v + 1]]
                    assert not any(u in ms and u != v for u in nb)


def test_library_local_order_equals_oracle():
    pytest = __import__("pytest")
    try:
        from paper_2205_03224_gb300 import local_order as lib_local_order, partition_geometric
        from paper_2205_03224_gb300 import _lib
        _lib.load()
    except (ImportError, OSError):
        pytest.skip("library not built")
    from oracle.partition import local_order
    for dims, nlev, p in (((13, 11, 9), 3, 8), ((20, 17), 3, 4), ((16, 16, 16), 4, 8)):
        A, xyz = gi.grid_operator(dims, beta=0.2)
        part = partition_geometric(A, xyz, nlev, p)
        for first in (0, 1, nlev - 1):
            ref = local_order(part, xyz, first)
            got = lib_local_order(part, xyz, first)
            assert np.array_equal(ref["perm"], got["perm"]), (dims, first)
