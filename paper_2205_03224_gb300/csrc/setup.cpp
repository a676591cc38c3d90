// Host-side setup of the GeMSLR hierarchy (Alg. 1 without the low-rank terms):
// symmetric permutation A_hat = P^T A P (eq. A0), slicing of B_l, E_l, F_l per
// level (Sec. 2.4), incomplete LU of every diagonal block of B_l and of the
// last-level blocks (Sec. 2.3, Sec. 4.3), and level-set analysis of the
// triangular factors for the GPU substitutions.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <exception>
#include <numeric>
#include <thread>

#include "internal.h"

namespace gemslr {

void fail(gemslr_status st, const std::string &msg) { throw Error{st, msg}; }

std::vector<double> splitmix_uniform01(uint64_t seed, int64_t count) {
    std::vector<double> v(count);
    uint64_t state = seed;
    for (int64_t i = 0; i < count; ++i) {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
    return v;
}

Csr csr_from_abi(const gemslr_csr *A) {
    if (!A || A->n < 0 || (A->n > 0 && (!A->rowptr || !A->colind || !A->val)))
        fail(GEMSLR_ERR_ARG, "invalid CSR matrix");
    Csr M;
    M.nrows = M.ncols = A->n;
    M.rp.assign(A->rowptr, A->rowptr + A->n + 1);
    int64_t nnz = M.rp[A->n];
    if (M.rp[0] != 0 || nnz < 0) fail(GEMSLR_ERR_ARG, "CSR row pointer must start at 0");
    if (A->n > 0 && nnz == 0) fail(GEMSLR_ERR_ARG, "CSR matrix without entries");
    for (int64_t i = 0; i < A->n; ++i)
        if (M.rp[i + 1] < M.rp[i]) fail(GEMSLR_ERR_ARG, "CSR row pointer not monotone");
    M.ci.assign(A->colind, A->colind + nnz);
    M.v.assign(A->val, A->val + nnz);
    for (int64_t i = 0; i < A->n; ++i)
        for (int64_t p = M.rp[i]; p < M.rp[i + 1]; ++p) {
            if (M.ci[p] < 0 || M.ci[p] >= A->n) fail(GEMSLR_ERR_ARG, "CSR column out of range");
            if (p > M.rp[i] && M.ci[p] <= M.ci[p - 1])
                fail(GEMSLR_ERR_ARG, "CSR columns must be strictly ascending");
        }
    return M;
}

Csr csr_from_mat(const gemslr_mat &m) {
    Csr M;
    M.nrows = m.nrows;
    M.ncols = m.ncols;
    if (m.nrows < 0 || m.ncols < 0 || (m.nrows > 0 && !m.rowptr))
        fail(GEMSLR_ERR_ARG, "invalid factor matrix");
    if (m.nrows == 0) return M;
    M.rp.assign(m.rowptr, m.rowptr + m.nrows + 1);
    int64_t nnz = M.rp[m.nrows];
    if (nnz > 0 && (!m.colind || !m.val)) fail(GEMSLR_ERR_ARG, "invalid factor matrix");
    M.ci.assign(m.colind, m.colind + nnz);
    M.v.assign(m.val, m.val + nnz);
    for (int64_t p = 0; p < nnz; ++p)
        if (M.ci[p] < 0 || M.ci[p] >= m.ncols) fail(GEMSLR_ERR_ARG, "factor column out of range");
    return M;
}

Csr permute_sym(const Csr &A, const std::vector<int32_t> &perm) {
    const int64_t n = A.nrows;
    std::vector<int32_t> inv(n);
    for (int64_t i = 0; i < n; ++i) inv[perm[i]] = (int32_t)i;
    Csr B;
    B.nrows = B.ncols = n;
    B.rp.assign(n + 1, 0);
    B.ci.resize(A.nnz());
    B.v.resize(A.nnz());
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = perm[i];
        row.clear();
        for (int64_t p = A.rp[o]; p < A.rp[o + 1]; ++p) row.emplace_back(inv[A.ci[p]], A.v[p]);
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                      return a.first < b.first;
                  });
        int64_t q = B.rp[i];
        for (auto &e : row) { B.ci[q] = e.first; B.v[q] = e.second; ++q; }
        B.rp[i + 1] = q;
    }
    return B;
}

Csr submatrix(const Csr &A, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
    Csr S;
    S.nrows = r1 - r0;
    S.ncols = c1 - c0;
    S.rp.assign(S.nrows + 1, 0);
    for (int64_t i = r0; i < r1; ++i) {
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
            int32_t c = A.ci[p];
            if (c >= c0 && c < c1) { S.ci.push_back((int32_t)(c - c0)); S.v.push_back(A.v[p]); }
        }
        S.rp[i - r0 + 1] = (int64_t)S.ci.size();
    }
    return S;
}

static std::vector<int64_t> block_of_rows(const std::vector<int64_t> &bp) {
    std::vector<int64_t> blk(bp.back());
    for (size_t j = 0; j + 1 < bp.size(); ++j)
        for (int64_t i = bp[j]; i < bp[j + 1]; ++i) blk[i] = (int64_t)j;
    return blk;
}

Csr block_diag_part(const Csr &A, const std::vector<int64_t> &bp) {
    std::vector<int64_t> blk = block_of_rows(bp);
    Csr S;
    S.nrows = A.nrows;
    S.ncols = A.ncols;
    S.rp.assign(A.nrows + 1, 0);
    for (int64_t i = 0; i < A.nrows; ++i) {
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
            if (blk[A.ci[p]] == blk[i]) { S.ci.push_back(A.ci[p]); S.v.push_back(A.v[p]); }
        S.rp[i + 1] = (int64_t)S.ci.size();
    }
    return S;
}

bool blocks_coupled(const Csr &A, const std::vector<int64_t> &bp) {
    std::vector<int64_t> blk = block_of_rows(bp);
    for (int64_t i = 0; i < A.nrows; ++i)
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
            if (blk[A.ci[p]] != blk[i]) return true;
    return false;
}

void append_block(Csr &dst, const Csr &blk, int64_t off) {
    for (int64_t i = 0; i < blk.nrows; ++i) {
        for (int64_t p = blk.rp[i]; p < blk.rp[i + 1]; ++p) {
            dst.ci.push_back((int32_t)(blk.ci[p] + off));
            dst.v.push_back(blk.v[p]);
            if (!blk.vi.empty()) dst.vi.push_back(blk.vi[p]);
        }
        dst.rp.push_back((int64_t)dst.ci.size());
    }
    dst.nrows += blk.nrows;
    dst.ncols += blk.ncols;
}

// ---- incomplete factorisations ---------------------------------------------
// The factorisations are written once for a scalar S: double, or
// std::complex<double> for the complex-shifted blocks B + i alpha I of
// Sec. 5.2.3 (values in v, imaginary parts in vi).  Every magnitude is the
// modulus |.|.
using zd = std::complex<double>;

template <typename S> S value_of(const Csr &B, int64_t p);
template <> double value_of<double>(const Csr &B, int64_t p) { return B.v[p]; }
template <> zd value_of<zd>(const Csr &B, int64_t p) { return zd(B.v[p], B.vi.empty() ? 0.0 : B.vi[p]); }
static void push_value(Csr &M, double x) { M.v.push_back(x); }
static void push_value(Csr &M, zd x) { M.v.push_back(x.real()); M.vi.push_back(x.imag()); }
static double sq(double x) { return x * x; }
static double sq(zd x) { return x.real() * x.real() + x.imag() * x.imag(); }

// Pivot rule for the (undiscussed) small-pivot case: |u_ii| below
// 1e-12*||a_i||_2 is replaced by sign(u_ii)*1e-12*||a_i||_2 (+ for zero);
// an all-zero row gets 1.  A complex pivot keeps its phase.
static double guard_pivot(double u, double rownorm, int64_t &count) {
    if (rownorm == 0.0) {
        if (u == 0.0) { ++count; return 1.0; }
        return u;
    }
    const double floor_ = 1e-12 * rownorm;
    if (std::fabs(u) < floor_) { ++count; return u < 0.0 ? -floor_ : floor_; }
    return u;
}
static zd guard_pivot(zd u, double rownorm, int64_t &count) {
    if (rownorm == 0.0) {
        if (u == 0.0) { ++count; return 1.0; }
        return u;
    }
    const double floor_ = 1e-12 * rownorm, a = std::abs(u);
    if (a < floor_) { ++count; return u == 0.0 ? zd(floor_) : u * (floor_ / a); }
    return u;
}

template <typename S>
static double norm2_row(const Csr &B, int64_t i) {
    double acc = 0.0;
    for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) acc += sq(value_of<S>(B, p));
    return std::sqrt(acc);
}

static void reset_factor(Csr &M, int64_t n) {
    M.nrows = M.ncols = n;
    M.rp.assign(1, 0);
    M.ci.clear();
    M.v.clear();
    M.vi.clear();
}

// ILU(0): elimination restricted to the pattern of B, rows top to bottom,
// multipliers in ascending column order (IKJ form).
template <typename S>
static int64_t ilu0_impl(const Csr &B, Csr &L, Csr &U) {
    const int64_t n = B.nrows;
    reset_factor(L, n);
    reset_factor(U, n);
    std::vector<S> row(n, S(0.0)), piv(n, S(0.0));
    std::vector<int64_t> stamp(n, -1);
    int64_t clamped = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) { row[B.ci[p]] = value_of<S>(B, p); stamp[B.ci[p]] = i; }
        for (int64_t p = B.rp[i]; p < B.rp[i + 1] && B.ci[p] < i; ++p) {
            const int32_t k = B.ci[p];
            row[k] = row[k] / piv[k];
            const S lik = row[k];
            for (int64_t q = U.rp[k] + 1; q < U.rp[k + 1]; ++q) {   // skip u_kk (first)
                const int32_t j = U.ci[q];
                if (stamp[j] == i) row[j] -= lik * value_of<S>(U, q);
            }
        }
        bool diag = false;
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) diag |= (B.ci[p] == i);
        const S d = guard_pivot(diag ? row[i] : S(0.0), norm2_row<S>(B, i), clamped);
        piv[i] = d;
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
            if (B.ci[p] < i) { L.ci.push_back(B.ci[p]); push_value(L, row[B.ci[p]]); }
        U.ci.push_back((int32_t)i);
        push_value(U, d);
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
            if (B.ci[p] > i) { U.ci.push_back(B.ci[p]); push_value(U, row[B.ci[p]]); }
        L.rp.push_back((int64_t)L.ci.size());
        U.rp.push_back((int64_t)U.ci.size());
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) row[B.ci[p]] = S(0.0);
    }
    return clamped;
}

// ILUT(tau, lfil), dual threshold.  Every candidate is measured in the units
// of the row being reduced (scale-independent reading): a multiplier l_ik by
// |l_ik * u_kk|, a U entry by |u_ij|; threshold tau*||a_i||_2; then the lfil
// largest of each part are kept (ties: lower column), the diagonal always.
template <typename S>
static int64_t ilut_impl(const Csr &B, double tau, int lfil, Csr &L, Csr &U) {
    const int64_t n = B.nrows;
    reset_factor(L, n);
    reset_factor(U, n);
    std::vector<S> row(n, S(0.0)), piv(n, S(0.0));
    std::vector<char> present(n, 0), eliminated(n, 0);
    std::vector<int32_t> cols;
    struct Cand { int32_t c; double mag; };
    std::vector<Cand> cand;
    auto by_size = [](const Cand &a, const Cand &b) {
        if (a.mag != b.mag) return a.mag > b.mag;
        return a.c < b.c;
    };
    auto by_col = [](const Cand &a, const Cand &b) { return a.c < b.c; };
    int64_t clamped = 0;
    for (int64_t i = 0; i < n; ++i) {
        cols.clear();
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) {
            row[B.ci[p]] = value_of<S>(B, p);
            if (!present[B.ci[p]]) { present[B.ci[p]] = 1; cols.push_back(B.ci[p]); }
        }
        const double thr = tau * norm2_row<S>(B, i);
        while (true) {   // smallest not-yet-eliminated column below the diagonal
            int32_t k = -1;
            for (int32_t c : cols)
                if (c < i && !eliminated[c] && (k < 0 || c < k)) k = c;
            if (k < 0) break;
            eliminated[k] = 1;
            if (std::abs(row[k]) < thr) { row[k] = S(0.0); continue; }
            row[k] = row[k] / piv[k];
            const S lik = row[k];
            for (int64_t q = U.rp[k] + 1; q < U.rp[k + 1]; ++q) {
                const int32_t j = U.ci[q];
                if (!present[j]) { present[j] = 1; row[j] = S(0.0); cols.push_back(j); }
                row[j] -= lik * value_of<S>(U, q);
            }
        }
        cand.clear();
        for (int32_t c : cols)
            if (c < i && row[c] != S(0.0) && std::abs(row[c] * piv[c]) >= thr)
                cand.push_back({c, std::abs(row[c] * piv[c])});
        if (lfil >= 0 && (int64_t)cand.size() > lfil) {
            std::sort(cand.begin(), cand.end(), by_size);
            cand.resize(lfil);
        }
        std::sort(cand.begin(), cand.end(), by_col);
        for (auto &e : cand) { L.ci.push_back(e.c); push_value(L, row[e.c]); }
        const S d = guard_pivot(present[i] ? row[i] : S(0.0), norm2_row<S>(B, i), clamped);
        piv[i] = d;
        U.ci.push_back((int32_t)i);
        push_value(U, d);
        cand.clear();
        for (int32_t c : cols)
            if (c > i && row[c] != S(0.0) && std::abs(row[c]) >= thr) cand.push_back({c, std::abs(row[c])});
        if (lfil >= 0 && (int64_t)cand.size() > lfil) {
            std::sort(cand.begin(), cand.end(), by_size);
            cand.resize(lfil);
        }
        std::sort(cand.begin(), cand.end(), by_col);
        for (auto &e : cand) { U.ci.push_back(e.c); push_value(U, row[e.c]); }
        L.rp.push_back((int64_t)L.ci.size());
        U.rp.push_back((int64_t)U.ci.size());
        for (int32_t c : cols) { row[c] = S(0.0); present[c] = 0; eliminated[c] = 0; }
    }
    return clamped;
}

int64_t factor_ilu0(const Csr &B, Csr &L, Csr &U) {
    return B.vi.empty() ? ilu0_impl<double>(B, L, U) : ilu0_impl<zd>(B, L, U);
}

int64_t factor_ilut(const Csr &B, double tau, int lfil, Csr &L, Csr &U) {
    return B.vi.empty() ? ilut_impl<double>(B, tau, lfil, L, U) : ilut_impl<zd>(B, tau, lfil, L, U);
}

// B + i alpha I of one block (Sec. 5.2.3): imaginary parts alpha on the
// diagonal (an entry is inserted where the pattern has none), 0 elsewhere.
static Csr shifted_block(const Csr &B, double alpha) {
    Csr S;
    S.nrows = B.nrows;
    S.ncols = B.ncols;
    S.rp.assign(1, 0);
    for (int64_t i = 0; i < B.nrows; ++i) {
        bool diag = false;
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) {
            if (!diag && B.ci[p] > i) {
                S.ci.push_back((int32_t)i);
                S.v.push_back(0.0);
                S.vi.push_back(alpha);
                diag = true;
            }
            S.ci.push_back(B.ci[p]);
            S.v.push_back(B.v[p]);
            S.vi.push_back(B.ci[p] == i ? alpha : 0.0);
            diag |= (B.ci[p] == i);
        }
        if (!diag) {
            S.ci.push_back((int32_t)i);
            S.v.push_back(0.0);
            S.vi.push_back(alpha);
        }
        S.rp.push_back((int64_t)S.ci.size());
    }
    return S;
}

// ---- level sets ------------------------------------------------------------
std::vector<int32_t> wavefronts_lower(const Csr &L, int64_t r0, int64_t r1) {
    std::vector<int32_t> lev(r1 - r0, 0);
    for (int64_t i = r0; i < r1; ++i) {
        int32_t m = 0;
        for (int64_t p = L.rp[i]; p < L.rp[i + 1]; ++p)
            m = std::max(m, lev[L.ci[p] - r0] + 1);
        lev[i - r0] = m;
    }
    return lev;
}

std::vector<int32_t> wavefronts_upper(const Csr &U, int64_t r0, int64_t r1) {
    std::vector<int32_t> lev(r1 - r0, 0);
    for (int64_t i = r1 - 1; i >= r0; --i) {
        int32_t m = 0;
        for (int64_t p = U.rp[i]; p < U.rp[i + 1]; ++p)
            if (U.ci[p] != i) m = std::max(m, lev[U.ci[p] - r0] + 1);
        lev[i - r0] = m;
    }
    return lev;
}

// ---- hierarchy ------------------------------------------------------------
// The diagonal blocks of a level are independent (Sec. 4.2), so they are
// factored by a pool of host threads (blocks handed out in turn); the factors
// are appended in block order, so the result does not depend on the threads.
static void factor_level(const Csr &B, const std::vector<int64_t> &bp, const gemslr_options *opt, double alpha,
                         Csr &L, Csr &U, int64_t &clamped) {
    if (opt->ilu_kind == GEMSLR_ILU0_DEVICE || opt->ilu_kind == GEMSLR_ILUT_DEVICE) {
        if (alpha != 0.0) fail(GEMSLR_ERR_UNSUPPORTED, "the complex shift needs a host factorisation (ILU0 or ILUT)");
        if (opt->ilu_kind == GEMSLR_ILU0_DEVICE) {
            factor_level_ilu0_device(B, bp, L, U, clamped);
            return;
        }
        // a row too wide for the device kernel: the host ILUT below (same factors)
        if (factor_level_ilut_device(B, bp, opt->ilut_tau, opt->ilut_lfil, L, U, clamped)) return;
    }
    const int64_t n = B.nrows;
    const size_t nb = bp.size() - 1;
    std::vector<Csr> Ls(nb), Us(nb);
    std::vector<int64_t> cl(nb, 0);
    std::vector<std::exception_ptr> err(nb);
    std::atomic<size_t> next{0};
    std::atomic<bool> failed{false};
    auto work = [&] {
        for (size_t j; !failed.load() && (j = next.fetch_add(1)) < nb;) {
            try {
                Csr Bj = submatrix(B, bp[j], bp[j + 1], bp[j], bp[j + 1]);
                if (alpha != 0.0) Bj = shifted_block(Bj, alpha);
                if (opt->ilu_kind == GEMSLR_ILU0 || opt->ilu_kind == GEMSLR_ILU0_DEVICE)
                    cl[j] = factor_ilu0(Bj, Ls[j], Us[j]);
                else cl[j] = factor_ilut(Bj, opt->ilut_tau, opt->ilut_lfil, Ls[j], Us[j]);
            } catch (...) {
                err[j] = std::current_exception();
                failed = true;
            }
        }
    };
    const size_t hw = std::max<unsigned>(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>(nb, std::min<size_t>(hw, 32));
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
    L = Csr();
    U = Csr();
    for (size_t j = 0; j < nb; ++j) {
        append_block(L, Ls[j], bp[j]);
        append_block(U, Us[j], bp[j]);
        clamped += cl[j];
    }
    L.nrows = L.ncols = U.nrows = U.ncols = n;
}

static void read_partition(const gemslr_partition *part, int64_t n, Hierarchy &h,
                           std::vector<std::vector<int64_t>> &bps) {
    if (!part || part->nlev < 2 || part->nlev > GEMSLR_MAX_LEVELS || !part->perm ||
        !part->level_ptr || !part->nblk || !part->block_ptr)
        fail(GEMSLR_ERR_ARG, "invalid partition (need 2 <= nlev <= 16 and all arrays)");
    h.nlev = part->nlev;
    h.perm.assign(part->perm, part->perm + n);
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (h.perm[i] < 0 || h.perm[i] >= n || seen[h.perm[i]])
            fail(GEMSLR_ERR_PARTITION, "perm is not a permutation");
        seen[h.perm[i]] = 1;
    }
    h.level_ptr.assign(part->level_ptr, part->level_ptr + h.nlev + 1);
    if (h.level_ptr[0] != 0 || h.level_ptr[h.nlev] != n)
        fail(GEMSLR_ERR_PARTITION, "level_ptr must run from 0 to n");
    int64_t off = 0;
    for (int l = 0; l < h.nlev; ++l) {
        if (h.level_ptr[l + 1] < h.level_ptr[l]) fail(GEMSLR_ERR_PARTITION, "level_ptr not monotone");
        int32_t nb = part->nblk[l];
        if (nb < 1) fail(GEMSLR_ERR_PARTITION, "every level needs at least one block");
        std::vector<int64_t> bp(part->block_ptr + off, part->block_ptr + off + nb + 1);
        off += nb + 1;
        if (bp[0] != 0 || bp[nb] != h.level_ptr[l + 1] - h.level_ptr[l])
            fail(GEMSLR_ERR_PARTITION, "block_ptr does not cover its level");
        for (int j = 0; j < nb; ++j)
            if (bp[j + 1] < bp[j]) fail(GEMSLR_ERR_PARTITION, "block_ptr not monotone");
        bps.push_back(bp);
    }
}

void build_levels(const Csr &A, const gemslr_partition *part, const gemslr_options *opt,
                  Hierarchy &h) {
    h.n = A.nrows;
    h.cplx = opt->shift != 0.0;
    h.alpha = 0.0;
    if (h.cplx) {   // alpha = shift * sum_i |a_ii| / n (Sec. 5.2.3)
        double sd = 0.0;
        for (int64_t i = 0; i < A.nrows; ++i)
            for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
                if (A.ci[p] == i) sd += std::fabs(A.v[p]);
        h.alpha = A.nrows ? opt->shift * sd / (double)A.nrows : 0.0;
    }
    std::vector<std::vector<int64_t>> bps;
    read_partition(part, h.n, h, bps);
    h.Ahat = permute_sym(A, h.perm);
    const int64_t n = h.n;
    h.lev.resize(h.nlev - 1);
    for (int l = 0; l < h.nlev - 1; ++l) {
        HostLevel &lv = h.lev[l];
        lv.s = h.level_ptr[l];
        lv.e = h.level_ptr[l + 1];
        lv.bp = bps[l];
        Csr B = submatrix(h.Ahat, lv.s, lv.e, lv.s, lv.e);
        if (blocks_coupled(B, lv.bp))
            fail(GEMSLR_ERR_PARTITION, "level " + std::to_string(l) + ": diagonal blocks are coupled");
        lv.E = submatrix(h.Ahat, lv.e, n, lv.s, lv.e);
        lv.F = submatrix(h.Ahat, lv.s, lv.e, lv.e, n);
        factor_level(B, lv.bp, opt, h.alpha, lv.L, lv.U, h.nclamp);
        lv.rank_req = opt->rank[l];
    }
    HostLevel &la = h.last;
    la.s = h.level_ptr[h.nlev - 1];
    la.e = n;
    la.bp = bps[h.nlev - 1];
    Csr C = block_diag_part(submatrix(h.Ahat, la.s, n, la.s, n), la.bp);
    factor_level(C, la.bp, opt, h.alpha, la.L, la.U, h.nclamp);
    if (opt->strict_pivots && h.nclamp > 0)
        fail(GEMSLR_ERR_ZERO_PIVOT, std::to_string(h.nclamp) + " pivots were clamped");
}

}  // namespace gemslr
