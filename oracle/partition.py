"""Multilevel p-way vertex-separator reordering (Alg. 3, Sec. 3.2).

The paper partitions |C_{l-1}| + |C_{l-1}^T| with ParMETIS.  The oracle uses a
geometric p-way partitioner that needs only the grid coordinates of the
unknowns:

  * recursive coordinate bisection (RCB) of the current vertex set S into p
    parts (p a power of two): split along the axis of largest extent (lowest
    axis on ties), ordering S by (coordinate, global index) and giving the
    first floor(|S|/2) vertices to the lower half of the part range;
  * separator = { v in S : some neighbour u of v inside S has
    part(u) < part(v) }.  For every edge between two parts the endpoint in
    the higher part is in the separator, so no edge joins two interiors
    (the vertex-separator definition of Sec. 3);
  * interior unknowns of part j (ascending global index) form block j of
    level l; the separator is the vertex set of level l+1 (Alg. 3 applies the
    partitioner to the subgraph induced by the separator).

The last level C_{L-2} is not partitioned: following Sec. 4.3 its unknowns
are ordered by reverse Cuthill-McKee on |C| + |C^T| and cut into p_last
contiguous chunks whose sizes differ by at most one (larger chunks first).

RCM reading: the paper only names RCM.  Here, per connected component in
order of discovery, the start vertex is an unvisited vertex of minimum
degree (lowest local index on ties); breadth-first search appends the
unvisited neighbours of each visited vertex sorted by (degree, local index);
the concatenated order is reversed.  Degrees count neighbours inside the set.

Output (all int64 unless noted):
  perm       new -> old, length n (int32)
  level_ptr  nlev + 1 offsets into perm
  nblk       blocks per level (int32)
  block_ptr  per level nblk[l]+1 offsets (relative to level_ptr[l]), concatenated
"""
from collections import deque

import numpy as np
import scipy.sparse as sp


def _sym_pattern(A):
    """Adjacency of |A| + |A^T| without the diagonal (CSR, sorted)."""
    S = sp.csr_matrix(A)
    P = (abs(S) + abs(S.T)).tocsr()
    P.setdiag(0)
    P.eliminate_zeros()
    P.sort_indices()
    return P


def rcb_parts(verts, coords, nparts):
    """Part number (0..nparts-1) of every vertex in ``verts`` (sorted global ids)."""
    part = np.zeros(len(verts), dtype=np.int64)

    def rec(idx, lo, np_):
        if np_ == 1 or len(idx) == 0:
            part[idx] = lo
            return
        c = coords[verts[idx]]
        ext = c.max(axis=0) - c.min(axis=0)
        ax = int(np.argmax(ext))            # first axis of largest extent
        order = np.lexsort((verts[idx], c[:, ax]))
        idx = idx[order]
        half = len(idx) // 2
        rec(idx[:half], lo, np_ // 2)
        rec(idx[half:], lo + np_ // 2, np_ - np_ // 2)

    rec(np.arange(len(verts)), 0, nparts)
    return part


def separator(verts, part, G):
    """Vertices of ``verts`` with a neighbour in the induced subgraph in a lower part."""
    n = G.shape[0]
    where = np.full(n, -1, dtype=np.int64)
    where[verts] = np.arange(len(verts))
    is_sep = np.zeros(len(verts), dtype=bool)
    for a, v in enumerate(verts):
        for u in G.indices[G.indptr[v]:G.indptr[v + 1]]:
            b = where[u]
            if b >= 0 and part[b] < part[a]:
                is_sep[a] = True
                break
    return is_sep


def rcm_order(G_local):
    """Reverse Cuthill-McKee order (local indices) of a symmetric pattern."""
    G = sp.csr_matrix(G_local)
    n = G.shape[0]
    deg = np.diff(G.indptr)
    visited = np.zeros(n, dtype=bool)
    order = []
    while len(order) < n:
        cand = np.flatnonzero(~visited)
        start = cand[np.lexsort((cand, deg[cand]))[0]]
        visited[start] = True
        q = deque([start])
        while q:
            v = q.popleft()
            order.append(v)
            nb = G.indices[G.indptr[v]:G.indptr[v + 1]]
            nb = nb[~visited[nb]]
            nb = nb[np.lexsort((nb, deg[nb]))]
            for u in nb:
                visited[u] = True
                q.append(u)
    return np.array(order[::-1], dtype=np.int64)


def multilevel_partition(A, coords, nlev, p, p_last=None):
    """Alg. 3 with the geometric p-way separator; ``nlev`` = Schur levels + last level."""
    p_last = p if p_last is None else p_last
    G = _sym_pattern(A)
    n = G.shape[0]
    coords = np.asarray(coords)
    verts = np.arange(n, dtype=np.int64)
    perm = []
    level_ptr = [0]
    nblk = []
    block_ptr = []
    for _ in range(nlev - 1):
        part = rcb_parts(verts, coords, p)
        is_sep = separator(verts, part, G)
        off = 0
        bp = [0]
        for j in range(p):
            blk = verts[(part == j) & ~is_sep]          # ascending global index
            perm.extend(blk.tolist())
            off += len(blk)
            bp.append(off)
        level_ptr.append(level_ptr[-1] + off)
        nblk.append(p)
        block_ptr.extend(bp)
        verts = verts[is_sep]
    # last level: RCM on the induced subgraph, p_last contiguous chunks
    sub = G[verts][:, verts]
    order = rcm_order(sub)
    perm.extend(verts[order].tolist())
    m = len(verts)
    sizes = [m // p_last + (1 if j < m % p_last else 0) for j in range(p_last)]
    bp = [0]
    for s in sizes:
        bp.append(bp[-1] + s)
    level_ptr.append(level_ptr[-1] + m)
    nblk.append(p_last)
    block_ptr.extend(bp)
    return dict(perm=np.array(perm, dtype=np.int32),
                level_ptr=np.array(level_ptr, dtype=np.int64),
                nblk=np.array(nblk, dtype=np.int32),
                block_ptr=np.array(block_ptr, dtype=np.int64))


def local_order(part, coords, first_level):
    """Local order inside the diagonal blocks (Sec. 3.2: each B_l may be permuted
    locally) of the levels first_level .. nlev-1.

    Reading: the vertices of a block are grouped into the 64 classes given by
    the parity of their 2 x 2 x 2 tile (floor(x/2), floor(y/2), floor(z/2) mod 2:
    tile colour t = tx + 2 ty + 4 tz) and the parity of the point itself (point
    colour c = px + 2 py + 4 pz); the classes are taken in the order of
    8 t + c, and inside a class the vertices keep their order.  Returns a copy
    of ``part`` with the new perm."""
    coords = np.asarray(coords, dtype=np.int64)
    perm = np.array(part["perm"], copy=True)
    nlev = len(part["nblk"])
    for l in range(first_level, nlev):
        _, _, bp = level_blocks(part, l)
        for j in range(len(bp) - 1):
            a, b = int(bp[j]), int(bp[j + 1])
            verts = perm[a:b]
            c = coords[verts]
            tile = ((c[:, 0] // 2) % 2) + 2 * ((c[:, 1] // 2) % 2) + 4 * ((c[:, 2] // 2) % 2)
            point = (c[:, 0] % 2) + 2 * (c[:, 1] % 2) + 4 * (c[:, 2] % 2)
            classes = 8 * tile + point
            out = []
            for k in range(64):                       # class after class, original order inside
                out.extend(verts[classes == k].tolist())
            perm[a:b] = out
    res = dict(part)
    res["perm"] = perm
    return res


def level_blocks(part, l):
    """(start, stop) offsets of level l and its block offsets (absolute)."""
    nblk = part["nblk"]
    off = int(sum(int(b) + 1 for b in nblk[:l]))
    bp = part["block_ptr"][off:off + int(nblk[l]) + 1] + part["level_ptr"][l]
    return int(part["level_ptr"][l]), int(part["level_ptr"][l + 1]), bp


def check_partition(A, part):
    """Raise if ``part`` is not a valid multilevel vertex-separator ordering.

    Checks that perm is a permutation, offsets are consistent, and that for
    every Schur level no edge of |A|+|A^T| joins two different blocks of the
    level (the blocks of B_l are uncoupled), Sec. 3.
    """
    n = A.shape[0]
    perm = part["perm"]
    if sorted(perm.tolist()) != list(range(n)):
        raise ValueError("perm is not a permutation")
    lp = part["level_ptr"]
    nlev = len(part["nblk"])
    if len(lp) != nlev + 1 or lp[0] != 0 or lp[-1] != n:
        raise ValueError("bad level_ptr")
    G = _sym_pattern(A)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    Gp = G[perm][:, perm].tocoo()
    for l in range(nlev - 1):
        s, e, bp = level_blocks(part, l)
        if bp[0] != s or bp[-1] != e:
            raise ValueError("bad block_ptr")
        blk = np.full(n, -1, dtype=np.int64)
        for j in range(len(bp) - 1):
            blk[bp[j]:bp[j + 1]] = j
        r, c = Gp.row, Gp.col
        mask = (r >= s) & (r < e) & (c >= s) & (c < e)
        if np.any(blk[r[mask]] != blk[c[mask]]):
            raise ValueError(f"level {l}: blocks are coupled")
    return True
