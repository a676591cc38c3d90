// Multilevel p-way vertex-separator reordering (Alg. 3, Sec. 3.2) with a
// geometric partitioner standing in for ParMETIS.
//
// Per Schur level the current vertex set S is cut into p parts by recursive
// coordinate bisection (axis of largest extent, lowest axis on ties; S ordered
// by (coordinate, global index); the first floor(|S|/2) vertices form the
// lower half of the part range).  A vertex with a neighbour of a lower part
// inside S joins the separator, which therefore separates the interiors
// (vertex-separator definition, Sec. 3); it becomes the next vertex set.
// The last level is ordered by reverse Cuthill-McKee on |C| + |C^T| (start:
// minimum degree, lowest index; neighbours visited by (degree, index)) and
// cut into p_last contiguous chunks whose sizes differ by at most one
// (Sec. 4.3).
#include <algorithm>
#include <cstdlib>
#include <deque>
#include <numeric>

#include "internal.h"

namespace gemslr {

namespace {

struct Graph {  // symmetric adjacency without self loops
    std::vector<int64_t> xadj;
    std::vector<int32_t> adj;
};

Graph symmetric_pattern(const Csr &A) {
    const int64_t n = A.nrows;
    std::vector<std::vector<int32_t>> nb(n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
            const int32_t j = A.ci[p];
            if (j == i || A.v[p] == 0.0) continue;
            nb[i].push_back(j);
            nb[j].push_back((int32_t)i);
        }
    Graph g;
    g.xadj.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        std::sort(nb[i].begin(), nb[i].end());
        nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
        g.xadj[i + 1] = g.xadj[i] + (int64_t)nb[i].size();
    }
    g.adj.reserve(g.xadj[n]);
    for (int64_t i = 0; i < n; ++i) g.adj.insert(g.adj.end(), nb[i].begin(), nb[i].end());
    return g;
}

void bisect(std::vector<int32_t> &ids, size_t a, size_t b, int lo, int np, const int32_t *xyz,
            std::vector<int32_t> &part_of) {
    if (np == 1 || a == b) {
        for (size_t t = a; t < b; ++t) part_of[ids[t]] = lo;
        return;
    }
    int32_t mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = xyz[3 * (int64_t)ids[a] + d]; mx[d] = mn[d]; }
    for (size_t t = a; t < b; ++t)
        for (int d = 0; d < 3; ++d) {
            mn[d] = std::min(mn[d], xyz[3 * (int64_t)ids[t] + d]);
            mx[d] = std::max(mx[d], xyz[3 * (int64_t)ids[t] + d]);
        }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
        if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
    std::sort(ids.begin() + a, ids.begin() + b, [&](int32_t u, int32_t v) {
        const int32_t cu = xyz[3 * (int64_t)u + ax], cv = xyz[3 * (int64_t)v + ax];
        return cu != cv ? cu < cv : u < v;
    });
    const size_t half = (b - a) / 2;
    bisect(ids, a, a + half, lo, np / 2, xyz, part_of);
    bisect(ids, a + half, b, lo + np / 2, np - np / 2, xyz, part_of);
}

std::vector<int32_t> reverse_cuthill_mckee(const Graph &g, const std::vector<int32_t> &verts) {
    const int64_t m = (int64_t)verts.size();
    std::vector<int64_t> local(g.xadj.size() - 1, -1);
    for (int64_t t = 0; t < m; ++t) local[verts[t]] = t;
    std::vector<std::vector<int32_t>> nb(m);
    for (int64_t t = 0; t < m; ++t)
        for (int64_t p = g.xadj[verts[t]]; p < g.xadj[verts[t] + 1]; ++p)
            if (local[g.adj[p]] >= 0) nb[t].push_back((int32_t)local[g.adj[p]]);
    std::vector<int64_t> deg(m);
    for (int64_t t = 0; t < m; ++t) deg[t] = (int64_t)nb[t].size();
    std::vector<char> seen(m, 0);
    std::vector<int32_t> order;
    order.reserve(m);
    while ((int64_t)order.size() < m) {
        int64_t start = -1;
        for (int64_t t = 0; t < m; ++t)
            if (!seen[t] && (start < 0 || deg[t] < deg[start])) start = t;
        seen[start] = 1;
        std::deque<int32_t> q{(int32_t)start};
        while (!q.empty()) {
            const int32_t v = q.front();
            q.pop_front();
            order.push_back(v);
            std::vector<int32_t> next;
            for (int32_t u : nb[v])
                if (!seen[u]) next.push_back(u);
            std::sort(next.begin(), next.end(), [&](int32_t x, int32_t y) {
                return deg[x] != deg[y] ? deg[x] < deg[y] : x < y;
            });
            for (int32_t u : next) { seen[u] = 1; q.push_back(u); }
        }
    }
    std::reverse(order.begin(), order.end());
    std::vector<int32_t> out(m);
    for (int64_t t = 0; t < m; ++t) out[t] = verts[order[t]];
    return out;
}

}  // namespace

void partition_geometric(const Csr &A, const int32_t *coords, int nlev, int p, int p_last,
                         std::vector<int32_t> &perm, std::vector<int64_t> &level_ptr,
                         std::vector<int32_t> &nblk, std::vector<int64_t> &block_ptr) {
    if (nlev < 2 || nlev > GEMSLR_MAX_LEVELS || p < 1 || (p & (p - 1)) != 0 || p_last < 1 || !coords)
        fail(GEMSLR_ERR_ARG, "partition: need 2 <= nlev <= 16, p a power of two, p_last >= 1");
    const int64_t n = A.nrows;
    Graph g = symmetric_pattern(A);
    std::vector<int32_t> verts(n);
    std::iota(verts.begin(), verts.end(), 0);
    std::vector<int32_t> part_of(n, -1);
    perm.clear();
    level_ptr.assign(1, 0);
    nblk.clear();
    block_ptr.clear();
    for (int l = 0; l + 1 < nlev; ++l) {
        std::vector<int32_t> ids = verts;
        bisect(ids, 0, ids.size(), 0, p, coords, part_of);
        std::vector<char> in_set(n, 0);
        for (int32_t v : verts) in_set[v] = 1;
        std::vector<char> sep(n, 0);
        for (int32_t v : verts)
            for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
                const int32_t u = g.adj[q];
                if (in_set[u] && part_of[u] < part_of[v]) { sep[v] = 1; break; }
            }
        std::vector<std::vector<int32_t>> blocks(p);
        std::vector<int32_t> next;
        for (int32_t v : verts) {   // verts ascending -> blocks ascending
            if (sep[v]) next.push_back(v);
            else blocks[part_of[v]].push_back(v);
        }
        int64_t off = 0;
        block_ptr.push_back(0);
        for (int j = 0; j < p; ++j) {
            perm.insert(perm.end(), blocks[j].begin(), blocks[j].end());
            off += (int64_t)blocks[j].size();
            block_ptr.push_back(off);
        }
        level_ptr.push_back(level_ptr.back() + off);
        nblk.push_back(p);
        verts.swap(next);
    }
    std::vector<int32_t> last = reverse_cuthill_mckee(g, verts);
    perm.insert(perm.end(), last.begin(), last.end());
    const int64_t m = (int64_t)last.size();
    block_ptr.push_back(0);
    int64_t off = 0;
    for (int j = 0; j < p_last; ++j) {
        off += m / p_last + (j < m % p_last ? 1 : 0);
        block_ptr.push_back(off);
    }
    level_ptr.push_back(level_ptr.back() + m);
    nblk.push_back(p_last);
}

// Local order inside the blocks of levels first .. nlev-1 (Sec. 3.2: each B_l
// may be permuted locally).  A block's vertices are sorted stably by the
// colour key 8 t + c, with t = (floor(x/2) mod 2) + 2 (floor(y/2) mod 2) +
// 4 (floor(z/2) mod 2) the colour of the vertex's 2 x 2 x 2 tile and
// c = (x mod 2) + 2 (y mod 2) + 4 (z mod 2) its point colour.  Two vertices of
// one class differ by an even amount in every coordinate, so no class holds
// two 7-point (or 5-point) neighbours: the classes are independent sets,
// which shortens the wavefronts of the blocks' triangular factors.
void local_order(const int32_t *coords, int64_t n, const std::vector<int64_t> &level_ptr,
                 const std::vector<int32_t> &nblk, const std::vector<int64_t> &block_ptr, int first,
                 std::vector<int32_t> &perm) {
    const int nlev = (int)nblk.size();
    if (first < 0 || first > nlev) fail(GEMSLR_ERR_ARG, "local order: first level out of range");
    auto key = [&](int32_t v) {
        const int32_t x = coords[3 * (int64_t)v], y = coords[3 * (int64_t)v + 1], z = coords[3 * (int64_t)v + 2];
        const int t = ((x >> 1) & 1) + 2 * ((y >> 1) & 1) + 4 * ((z >> 1) & 1);
        const int c = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
        return 8 * t + c;
    };
    int64_t off = 0;
    for (int l = 0; l < nlev; ++l) {
        for (int j = 0; j < nblk[l]; ++j) {
            if (l < first) continue;
            const int64_t a = level_ptr[l] + block_ptr[off + j], b = level_ptr[l] + block_ptr[off + j + 1];
            if (a < 0 || b > n || a > b) fail(GEMSLR_ERR_PARTITION, "local order: block out of range");
            std::stable_sort(perm.begin() + a, perm.begin() + b,
                             [&](int32_t u, int32_t v) { return key(u) < key(v); });
        }
        off += nblk[l] + 1;
    }
}

}  // namespace gemslr
