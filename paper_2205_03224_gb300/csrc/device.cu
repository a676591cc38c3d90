// Device layout of the GeMSLR hierarchy and the application of M^{-1} (Alg. 2).
#include <algorithm>
#include <complex>
#include <atomic>
#include <cstring>
#include <mutex>

#include "device.h"

namespace gemslr {

void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) fail(GEMSLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- instrumentation ---------------------------------------------------------
namespace {
struct ProfEntry { std::string name; cudaEvent_t a, b; };
struct ProfStat { double ms = 0.0; int64_t count = 0; };
std::atomic<uint64_t> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfEntry> g_prof_pending;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_pool;
std::vector<std::pair<std::string, ProfStat>> g_prof_stats;
}  // namespace

void count_launch(int n) { g_launches += (uint64_t)n; }

bool profile_enabled() { return g_prof_on; }

ProfScope::ProfScope(const char *name, cudaStream_t s) : slot(-1), st(s) {
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::pair<cudaEvent_t, cudaEvent_t> ev;
    if (!g_prof_pool.empty()) { ev = g_prof_pool.back(); g_prof_pool.pop_back(); }
    else { cudaEventCreate(&ev.first); cudaEventCreate(&ev.second); }
    cudaEventRecord(ev.first, st);
    g_prof_pending.push_back({name, ev.first, ev.second});
    slot = (int)g_prof_pending.size() - 1;
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof_pending[slot].b, st);
}

void profile_enable(bool on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on;
}

// Synchronise the recorded events and fold them into the per-name totals.
void profile_collect() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &e : g_prof_pending) {
        cudaEventSynchronize(e.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.a, e.b);
        auto it = std::find_if(g_prof_stats.begin(), g_prof_stats.end(),
                               [&](const std::pair<std::string, ProfStat> &p) { return p.first == e.name; });
        if (it == g_prof_stats.end()) { g_prof_stats.push_back({e.name, ProfStat()}); it = g_prof_stats.end() - 1; }
        it->second.ms += ms;
        it->second.count += 1;
        g_prof_pool.push_back({e.a, e.b});
    }
    g_prof_pending.clear();
}

void profile_reset() {
    profile_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_stats.clear();
}

int profile_read(char *names, size_t len, double *ms, int64_t *counts, int maxn) {
    profile_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::string all;
    int k = 0;
    for (auto &p : g_prof_stats) {
        if (k < maxn) {
            if (ms) ms[k] = p.second.ms;
            if (counts) counts[k] = p.second.count;
        }
        all += p.first;
        all += '\n';
        ++k;
    }
    if (names && len) {
        const size_t c = std::min(len - 1, all.size());
        std::memcpy(names, all.data(), c);
        names[c] = 0;
    }
    return k;
}

uint64_t launches_total() { return g_launches.load(); }

Arena::~Arena() {
    // cudaFree waits for the device; a caller's allocator may hand the memory
    // out again at once, so the handle's work must be finished first
    if (free_fn_ && !ptrs_.empty()) cudaDeviceSynchronize();
    for (void *p : ptrs_) {
        if (free_fn_) free_fn_(p, ctx_);
        else cudaFree(p);
    }
}

void *Arena::alloc(size_t bytes) {
    void *p = nullptr;
    const size_t b = bytes ? (bytes + 255) & ~size_t(255) : 256;
    if (alloc_fn_) {
        p = alloc_fn_(b, ctx_);
        if (!p) fail(GEMSLR_ERR_NOMEM, "device allocation of " + std::to_string(b) + " bytes failed (caller's allocator)");
        if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
            free_fn_(p, ctx_);
            fail(GEMSLR_ERR_ARG, "caller's allocator returned a pointer not aligned to 256 bytes");
        }
    } else if (cudaMalloc(&p, b) != cudaSuccess) {
        cudaGetLastError();
        fail(GEMSLR_ERR_NOMEM, "device allocation of " + std::to_string(b) + " bytes failed");
    }
    ptrs_.push_back(p);
    total_ += b;
    return p;
}

namespace {


// Every entry must lie in its row's diagonal block, strictly below (L) or on
// and above (U) the diagonal, and U needs a nonzero diagonal: the kernels
// index the block's shared-memory vector with these columns.
void validate_tri(const Csr &T, const std::vector<int64_t> &bp, bool upper) {
    if (T.nrows != bp.back()) fail(GEMSLR_ERR_ARG, "factor rows do not match the level");
    for (size_t b = 0; b + 1 < bp.size(); ++b)
        for (int64_t i = bp[b]; i < bp[b + 1]; ++i) {
            bool diag = false;
            for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p) {
                const int64_t c = T.ci[p];
                if (c < bp[b] || c >= bp[b + 1]) fail(GEMSLR_ERR_ARG, "factor entry outside its diagonal block");
                if (!upper && c >= i) fail(GEMSLR_ERR_ARG, "L must be strictly lower triangular");
                if (upper && c < i) fail(GEMSLR_ERR_ARG, "U must be upper triangular");
                if (upper && c == i) diag = T.v[p] != 0.0 || (!T.vi.empty() && T.vi[p] != 0.0);
            }
            if (upper && !diag) fail(GEMSLR_ERR_ARG, "U needs a nonzero diagonal");
        }
}

size_t pad16(size_t x) { return (x + 15) & ~size_t(15); }

// Entry p of a factor (and the reciprocal of a diagonal entry) in the value
// type of the substitution; complex factors keep their imaginary parts in vi.
template <typename VT> VT entry_at(const Csr &T, int64_t p) { return cast_to<VT>(T.v[p]); }
template <> zc entry_at<zc>(const Csr &T, int64_t p) { return zc(T.v[p], T.vi.empty() ? 0.0 : T.vi[p]); }
template <typename VT> VT inv_entry(const Csr &T, int64_t p) { return cast_to<VT>(1.0 / T.v[p]); }
template <> zc inv_entry<zc>(const Csr &T, int64_t p) {
    const std::complex<double> r = 1.0 / std::complex<double>(T.v[p], T.vi.empty() ? 0.0 : T.vi[p]);
    return zc(r.real(), r.imag());
}
// The stored value of an off-diagonal entry: -t_ij (L, pdiag < 0) or
// -u_ij / u_ii (U, u_ii at pdiag), formed in FP64 and rounded once.
template <typename VT> VT stored_entry(const Csr &T, int64_t p, int64_t pdiag) {
    return cast_to<VT>(pdiag < 0 ? -T.v[p] : -(T.v[p] * (1.0 / T.v[pdiag])));
}
template <> zc stored_entry<zc>(const Csr &T, int64_t p, int64_t pdiag) {
    const zc v = entry_at<zc>(T, p);
    return pdiag < 0 ? -v : -(v * inv_entry<zc>(T, pdiag));
}

}  // namespace

template <typename VT>
int64_t chunk_slots(int64_t maxlen) {
    return LanesPerRow<VT>::value == 1 ? maxlen : 4 * ((maxlen + 3) / 4);
}

template <typename VT>
size_t chunk_bytes(int64_t nrows, int64_t maxlen, bool upper) {
    const size_t pr = (size_t)((nrows + 3) & ~int64_t(3));
    const size_t ne = (size_t)(chunk_slots<VT>(maxlen) * nrows);
    return 16 + 8 * pr + pad16(ne * 4) + pad16(ne * sizeof(VT)) + (upper ? pad16((size_t)nrows * sizeof(VT)) : 0);
}

// Append the chunks of one triangular factor of block [r0, r1) (see kernels.cuh).
template <typename VT>
void append_factor_chunks(const Csr &T, int64_t r0, int64_t r1, bool upper, ChunkHost<VT> &out, int &maxwf,
                          int max_rows, int stage_bytes) {
    std::vector<int32_t> lev = upper ? wavefronts_upper(T, r0, r1) : wavefronts_lower(T, r0, r1);
    int nw = 0;
    for (int32_t x : lev) nw = std::max(nw, x + 1);
    maxwf = std::max(maxwf, nw);
    std::vector<std::vector<int64_t>> rows(nw);
    for (int64_t i = r0; i < r1; ++i) rows[lev[i - r0]].push_back(i);
    std::vector<int64_t> nlen(r1 - r0);
    for (int64_t i = r0; i < r1; ++i) {
        int64_t c = 0;
        for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p) c += (T.ci[p] != i);
        nlen[i - r0] = c;
    }
    for (int w = 0; w < nw; ++w) {
        std::vector<int64_t> &R = rows[w];
        std::stable_sort(R.begin(), R.end(), [&](int64_t a, int64_t c) { return nlen[a - r0] > nlen[c - r0]; });
        if (!upper && nlen[R[0] - r0] == 0) continue;          // rows without L entries: x_i unchanged
        size_t start = 0;
        while (start < R.size()) {
            const int64_t maxlen = nlen[R[start] - r0];
            int64_t n = 0;
            while (start + n < R.size() && n < max_rows &&
                   chunk_bytes<VT>(n + 1, maxlen, upper) <= (size_t)stage_bytes)
                ++n;
            if (n == 0) fail(GEMSLR_ERR_UNSUPPORTED, "a factor row has too many entries for the staged substitution");
            const size_t bytes = chunk_bytes<VT>(n, maxlen, upper);
            const int64_t S = chunk_slots<VT>(maxlen);
            out.max_slots = std::max(out.max_slots, (int)S);
            const size_t base = out.data.size();
            out.data.resize(base + bytes, 0);
            unsigned char *p = out.data.data() + base;
            int32_t *hdr = reinterpret_cast<int32_t *>(p);
            hdr[0] = (int32_t)n;
            hdr[1] = (int32_t)S;
            hdr[2] = upper ? 1 : 0;
            hdr[3] = 0;                                          // slices that follow in the chunk
            const int64_t pr = (n + 3) & ~int64_t(3);
            int32_t *rr = hdr + 4, *ll = rr + pr, *cc = ll + pr;
            VT *vv = reinterpret_cast<VT *>(reinterpret_cast<unsigned char *>(cc) + pad16((size_t)(S * n) * 4));
            VT *dd = reinterpret_cast<VT *>(reinterpret_cast<unsigned char *>(vv) + pad16((size_t)(S * n) * sizeof(VT)));
            // the chunks store -t_ij (L) and -u_ij / u_ii (U), so that a row is
            // x_i (times 1/u_ii) plus one sum of products (see kernels.cuh)
            for (int64_t t = 0; t < n; ++t) {
                const int64_t i = R[start + t];
                rr[t] = (int32_t)(i - r0);
                ll[t] = (int32_t)nlen[i - r0];
                int64_t pdiag = -1;
                if (upper)
                    for (int64_t pp = T.rp[i]; pp < T.rp[i + 1]; ++pp)
                        if (T.ci[pp] == i) pdiag = pp;
                if (upper) dd[t] = inv_entry<VT>(T, pdiag);
                int64_t q = 0;
                for (int64_t pp = T.rp[i]; pp < T.rp[i + 1]; ++pp) {
                    if (T.ci[pp] == i) continue;
                    const int64_t e = LanesPerRow<VT>::value == 1 ? q * n + t : ((q >> 2) * n + t) * 4 + (q & 3);
                    cc[e] = (int32_t)(T.ci[pp] - r0);
                    vv[e] = stored_entry<VT>(T, pp, pdiag);
                    ++q;
                }
            }
            {   // the kernels find a chunk in its group from the sizes of the chunks before it
                const size_t pr4 = (size_t)((hdr[0] + 3) & ~3), ne4 = (size_t)hdr[1] * (size_t)hdr[0];
                const size_t dev = 16 + 8 * pr4 + pad16(ne4 * 4) + pad16(ne4 * sizeof(VT)) +
                                   (hdr[2] ? pad16((size_t)hdr[0] * sizeof(VT)) : 0);
                if (dev != bytes) fail(GEMSLR_ERR_ARG, "chunk header does not describe its size");
            }
            out.off.push_back((int64_t)out.data.size());
            start += n;
        }
    }
}

template <typename VT>
void build_chunks(const Csr &L, const Csr &U, const std::vector<int64_t> &bp, ChunkHost<VT> &out, int max_rows,
                  int max_slices, int stage_bytes) {
    if (max_slices < 1 || max_slices > kMaxSlices) fail(GEMSLR_ERR_ARG, "slices per chunk out of range");
    validate_tri(L, bp, false);
    validate_tri(U, bp, true);
    for (size_t b = 0; b + 1 < bp.size(); ++b) {
        const size_t first = out.off.size() - 1;
        append_factor_chunks<VT>(L, bp[b], bp[b + 1], false, out, out.maxwf_L, max_rows, stage_bytes);
        append_factor_chunks<VT>(U, bp[b], bp[b + 1], true, out, out.maxwf_U, max_rows, stage_bytes);
        if (max_slices >= 2) {
            // join up to max_slices consecutive slices into one chunk (<= stage_bytes)
            // by dropping the boundaries between them; the header of every slice but
            // the chunk's last says that another one follows
            std::vector<int64_t> keep(out.off.begin(), out.off.begin() + (int64_t)first + 1);
            size_t c = first;
            const size_t last = out.off.size() - 1;
            while (c < last) {
                const int64_t a0 = out.off[c];
                size_t e = c + 1;                    // slices [c, e) form the chunk
                while (e < last && (int)(e + 1 - c) <= max_slices && out.off[e + 1] - a0 <= (int64_t)stage_bytes) ++e;
                for (size_t t = c; t + 1 < e; ++t) reinterpret_cast<int32_t *>(out.data.data() + out.off[t])[3] = 1;
                keep.push_back(out.off[e]);
                c = e;
            }
            out.off.swap(keep);
        }
        out.blk_chunk.push_back((int32_t)(out.off.size() - 1));
    }
    if (out.data.empty()) out.data.resize(16, 0);
}


template void build_chunks<float>(const Csr &, const Csr &, const std::vector<int64_t> &, ChunkHost<float> &, int, int,
                                  int);
template void build_chunks<double>(const Csr &, const Csr &, const std::vector<int64_t> &, ChunkHost<double> &, int,
                                   int, int);
template void build_chunks<zc>(const Csr &, const Csr &, const std::vector<int64_t> &, ChunkHost<zc> &, int, int, int);

namespace {


template <typename VT, typename WT>
void upload_level(const HostLevel &hl, int64_t n, bool schur, Arena &a, DevLevel<VT, WT> &d, int smem_limit) {
    LevelView<VT, WT> &v = d.view;
    v.s = hl.s;
    v.e = hl.e;
    v.stail = schur ? n - hl.e : 0;
    v.nblk = (int32_t)hl.bp.size() - 1;
    v.blk_row = a.upload(hl.bp);
    int64_t maxrows = 0;
    for (size_t b = 0; b + 1 < hl.bp.size(); ++b) maxrows = std::max(maxrows, hl.bp[b + 1] - hl.bp[b]);
    d.smem_rows = (kRingBytes + maxrows * (int64_t)sizeof(VT) <= smem_limit) ? (int)maxrows : 0;
    ChunkHost<VT> ch;
    build_chunks<VT>(hl.L, hl.U, hl.bp, ch, kChunkRows, LanesPerRow<VT>::value == 1 ? kMaxSlices : 1,
                     StageBytesOf<VT>::value);
    v.C.data = a.upload(ch.data);
    v.C.off = a.upload(ch.off);
    v.C.blk_chunk = a.upload(ch.blk_chunk);
    v.max_slots = ch.max_slots;
    d.nwf_L = ch.maxwf_L;
    d.nwf_U = ch.maxwf_U;
    d.nchunks = (int64_t)ch.off.size() - 1;
    d.nnz_tri = hl.L.nnz() + hl.U.nnz();
    if (schur) {
        std::vector<int32_t> fci(hl.F.ci.size());
        for (size_t p = 0; p < fci.size(); ++p) fci[p] = (int32_t)(hl.F.ci[p] + hl.e);
        v.F_rp = a.upload(hl.F.rp);
        v.F_ci = a.upload(fci);
        v.F_v = a.upload(convert<VT>(hl.F.v));
        std::vector<int32_t> frows, fblk(1, 0);
        for (size_t b = 0; b + 1 < hl.bp.size(); ++b) {
            for (int64_t i = hl.bp[b]; i < hl.bp[b + 1]; ++i)
                if (hl.F.rp[i + 1] > hl.F.rp[i]) frows.push_back((int32_t)i);
            fblk.push_back((int32_t)frows.size());
        }
        if (frows.empty()) frows.push_back(0);
        v.F_rows = a.upload(frows);
        v.F_blk = a.upload(fblk);
        v.E_rp = a.upload(hl.E.rp);
        v.E_ci = a.upload(hl.E.ci);
        v.E_v = a.upload(convert<VT>(hl.E.v));
    }
    if (!schur) {
        v.F_rp = nullptr;
        v.F_ci = nullptr;
        v.F_v = nullptr;
        v.F_rows = nullptr;
        v.F_blk = nullptr;
    }
    v.k = 0;
    v.W = nullptr;
    v.H = nullptr;
}

}  // namespace

template <typename VT, typename WT>
void set_lowrank(DevLevel<VT, WT> &d, const HostLevel &hl, Arena &a) {
    d.view.k = hl.k;
    if (hl.k > 0) {
        d.view.W = a.upload(convert<WT>(hl.W));
        d.view.H = a.upload(convert<VT>(hl.H));
    }
}

// complex W, H: real parts in W, H and imaginary parts in Wi, Hi (empty: real)
template <>
void set_lowrank<zc, zc>(DevLevel<zc, zc> &d, const HostLevel &hl, Arena &a) {
    d.view.k = hl.k;
    if (hl.k > 0) {
        auto pack = [](const std::vector<double> &re, const std::vector<double> &im) {
            std::vector<zc> z(re.size());
            for (size_t i = 0; i < re.size(); ++i) z[i] = zc(re[i], im.empty() ? 0.0 : im[i]);
            return z;
        };
        d.view.W = a.upload(pack(hl.W, hl.Wi));
        d.view.H = a.upload(pack(hl.H, hl.Hi));
    }
}

template <typename VT, typename WT>
void upload_hierarchy(const Hierarchy &h, Arena &a, DevHierarchy<VT, WT> &d, int smem_limit) {
    set_trsv_smem_limit<VT, WT>(smem_limit);
    d.err = (int32_t *)a.alloc(sizeof(int32_t) * 4);
    GEMSLR_CUDA(cudaMemset(d.err, 0, sizeof(int32_t) * 4));
    d.lev.resize(h.lev.size());
    int64_t maxd = 1;
    for (size_t l = 0; l < h.lev.size(); ++l) {
        upload_level<VT, WT>(h.lev[l], h.n, true, a, d.lev[l], smem_limit);
        d.lev[l].view.err = d.err;
        set_lowrank<VT, WT>(d.lev[l], h.lev[l], a);
        maxd = std::max(maxd, h.lev[l].e - h.lev[l].s);
    }
    upload_level<VT, WT>(h.last, h.n, false, a, d.last, smem_limit);
    d.last.view.err = d.err;
    maxd = std::max(maxd, h.n - h.last.s);
    d.work = (VT *)a.alloc(sizeof(VT) * std::max<int64_t>(h.n, 1));
    d.scratch = (VT *)a.alloc(sizeof(VT) * maxd);
    int64_t maxgrid = 1;
    for (auto &l : h.lev) maxgrid = std::max(maxgrid, (h.n - l.e + kCoupleRows - 1) / kCoupleRows);
    d.partial = (VT *)a.alloc(sizeof(VT) * maxgrid * kMaxRank);
    d.counter = (unsigned *)a.alloc(sizeof(unsigned) * 4);
    GEMSLR_CUDA(cudaMemset(d.counter, 0, sizeof(unsigned) * 4));
    d.u = (VT *)a.alloc(sizeof(VT) * kMaxRank);
}

template <typename VT, typename WT>
void setup_inner(const Hierarchy &h, Arena &a, DevHierarchy<VT, WT> &d, int k, int sms) {
    DevInner<VT> &I = d.inner;
    if (k > 0 && !I.work2) {
        const int64_t e0 = h.lev[0].e, n = h.n, m = n - e0;
        // rows [e0, n) of A_hat with global columns, values in the application's precision
        const Csr &A = h.Ahat;
        std::vector<int64_t> rp(m + 1);
        for (int64_t i = 0; i <= m; ++i) rp[i] = A.rp[e0 + i] - A.rp[e0];
        std::vector<int32_t> ci(A.ci.begin() + A.rp[e0], A.ci.begin() + A.rp[n]);
        std::vector<double> v(A.v.begin() + A.rp[e0], A.v.begin() + A.rp[n]);
        InnerView<VT> &iv = I.iv;
        iv.m = m;
        iv.e0 = e0;
        iv.rp = a.upload(rp);
        iv.ci = a.upload(ci);
        iv.v = a.upload(convert<VT>(v));
        const size_t mm = (size_t)std::max<int64_t>(m, 1);
        iv.V = (VT *)a.alloc(sizeof(VT) * mm * (kMaxInner + 1));
        iv.Z = (VT *)a.alloc(sizeof(VT) * mm * kMaxInner);
        iv.w = (VT *)a.alloc(sizeof(VT) * mm);
        iv.H = (double *)a.alloc(sizeof(double) * (kMaxInner + 1) * kMaxInner);
        GEMSLR_CUDA(cudaMemset(iv.H, 0, sizeof(double) * (kMaxInner + 1) * kMaxInner));
        iv.grid = (int)std::max<int64_t>(1, std::min<int64_t>((m + kReduceThreads - 1) / kReduceThreads, 2 * sms));
        iv.partial = (double *)a.alloc(sizeof(double) * iv.grid * (kMaxInner + 2));
        iv.counter = (unsigned *)a.alloc(16);
        GEMSLR_CUDA(cudaMemset(iv.counter, 0, 16));
        iv.ctl = (InnerCtl *)a.alloc(sizeof(InnerCtl));
        GEMSLR_CUDA(cudaMemset(iv.ctl, 0, sizeof(InnerCtl)));
        I.work2 = (VT *)a.alloc(sizeof(VT) * std::max<int64_t>(n, 1));
        GEMSLR_CUDA(cudaMemset(I.work2, 0, sizeof(VT) * std::max<int64_t>(n, 1)));
        I.zero_rp = (int64_t *)a.alloc(sizeof(int64_t) * (mm + 1));
        GEMSLR_CUDA(cudaMemset(I.zero_rp, 0, sizeof(int64_t) * (mm + 1)));
    }
    I.k = k;
    I.iv.k = k;
}

// Alg. 2 at the root level with step 9: z1 = U^-1 L^-1 b1, z2 = b2 - E z1,
// k GMRES steps on S_hat_0 y2 = z2 (inner.cu) whose preconditioner is the
// level-0 correction plus the levels below, y1 = z1 - U^-1 L^-1 F y2.
template <typename VT, typename WT>
void apply_root_inner(DevHierarchy<VT, WT> &d, const IoT<VT> *in, VT *work, IoT<VT> *out_final, cudaStream_t st) {
    DevLevel<VT, WT> &L0 = d.lev[0];
    DevInner<VT> &I = d.inner;
    const InnerView<VT> &iv = I.iv;
    VT *work2 = I.work2;
    {
        ProfScope ps("trsv_down_L0", st);
        launch_trsv<VT, WT>(L0.view, 0, L0.smem_rows, in, work, nullptr, d.scratch, st);
    }
    LevelView<VT, WT> v0 = L0.view;
    v0.k = 0;                                       // z2 only: the correction acts inside the preconditioner
    {
        ProfScope ps("couple_EWt_L0", st);
        launch_couple<VT, WT>(v0, in, work, d.partial, d.counter, d.u, st);
    }
    {
        ProfScope ps("inner_start", st);
        launch_inner_norm<VT>(iv, work + iv.e0, st);
        launch_inner_start<VT>(iv, work + iv.e0, work2, st);
    }
    LevelView<VT, WT> vz = L0.view;
    vz.E_rp = I.zero_rp;                            // E_0 empty: z2 = v_j unchanged, u = H_0 W_0^T v_j
    PendingLowRank<VT, WT> pend;
    if (L0.view.k > 0 && L0.view.stail > 0) {
        pend.W = L0.view.W;
        pend.u = d.u;
        pend.ld = L0.view.stail;
        pend.row0 = L0.view.e;
        pend.k = L0.view.k;
    }
    for (int j = 0; j < I.k; ++j) {
        if (pend.W) {
            ProfScope ps("couple_EWt_L0", st);
            launch_couple<VT, WT>(vz, nullptr, work2, d.partial, d.counter, d.u, st);
        }
        apply_levels<VT, WT>(d, 1, nullptr, work2, nullptr, st, pend);   // z_j = M_S^-1 v_j in the tail
        {
            ProfScope ps("inner_trsv_L0", st);                              // level part: -U^-1 L^-1 F z_j
            launch_trsv<VT, WT>(L0.view, 1, L0.smem_rows, nullptr, work2, nullptr, d.scratch, st);
        }
        {
            ProfScope ps("inner_spmv_gs", st);
            launch_inner_spmv_dots<VT>(iv, j, work2, st);
            launch_inner_sub_dots<VT>(iv, j, st);
            launch_inner_scale<VT>(iv, j, work2, st);
        }
    }
    {
        ProfScope ps("inner_finish", st);
        launch_inner_lsq<VT>(iv, st);
        launch_inner_combine<VT>(iv, work, out_final, st);
    }
    {
        ProfScope ps("trsv_up_L0", st);
        launch_trsv<VT, WT>(L0.view, 1, L0.smem_rows, nullptr, work, out_final, d.scratch, st);
    }
}

template <typename VT, typename WT>
void apply_levels(DevHierarchy<VT, WT> &d, int from, const IoT<VT> *in, VT *work, IoT<VT> *out_final,
                  cudaStream_t st, const PendingLowRank<VT, WT> &pend0) {
    const int nl = (int)d.lev.size();
    constexpr bool kReal = !IsComplex<VT>::value;   // the complex hierarchy has neither inner steps nor a learned stage
    if constexpr (kReal) {
        if (from == 0 && nl >= 1 && d.inner.k > 0) {
            apply_root_inner<VT, WT>(d, in, work, out_final, st);
            return;
        }
    }
    static const char *kDown[] = {"trsv_down_L0", "trsv_down_L1", "trsv_down_L2", "trsv_down_L3", "trsv_down_L4+"};
    static const char *kUp[] = {"trsv_up_L0", "trsv_up_L1", "trsv_up_L2", "trsv_up_L3", "trsv_up_L4+"};
    static const char *kCouple[] = {"couple_EWt_L0", "couple_EWt_L1", "couple_EWt_L2", "couple_EWt_L3", "couple_EWt_L4+"};
    // learned correction at the deepest Schur level (active only when that level is part of this application)
    const bool learn = kReal && d.learned && d.learned->enabled && nl >= 1 && from <= nl - 1;
    // W_l u_l of the level before is added where its tail rows are first read
    PendingLowRank<VT, WT> pend = pend0;
    for (int l = from; l < nl; ++l) {
        DevLevel<VT, WT> &L = d.lev[l];
        const IoT<VT> *src = (l == from) ? in : nullptr;
        {
            ProfScope ps(kDown[std::min(l, 4)], st);
            launch_trsv<VT, WT>(L.view, 0, L.smem_rows, src, work, nullptr, d.scratch, st, pend);
        }
        {
            ProfScope ps(kCouple[std::min(l, 4)], st);
            launch_couple<VT, WT>(L.view, src, work, d.partial, d.counter, d.u, st, pend);
        }
        if constexpr (kReal)
            if (learn && l == nl - 1) learned_save<VT>(*d.learned, L.view.e, work, st);   // z2 of level l*
        pend = PendingLowRank<VT, WT>();
        if (L.view.k > 0 && L.view.stail > 0) {
            pend.W = L.view.W;
            pend.u = d.u;
            pend.ld = L.view.stail;
            pend.row0 = L.view.e;
            pend.k = L.view.k;
        }
    }
    {
        ProfScope ps("trsv_last", st);
        launch_trsv<VT, WT>(d.last.view, 0, d.last.smem_rows, from == nl ? in : nullptr, work,
                            learn ? nullptr : out_final, d.scratch, st, pend);
    }
    if constexpr (kReal) if (learn) {
        // S_hat y2 = C y2 - E (LU)^{-1} F y2 on a scratch vector, then y2 += N(rho)
        ProfScope ps("learned_stage", st);
        DevLevel<VT, WT> &L = d.lev[nl - 1];
        LearnedStage<VT> &Ls = *d.learned;
        const int64_t e = L.view.e, s0 = L.view.s, ntail = L.view.stail;
        GEMSLR_CUDA(cudaMemcpyAsync(Ls.work2 + e, work + e, sizeof(VT) * ntail, cudaMemcpyDeviceToDevice, st));
        GEMSLR_CUDA(cudaMemsetAsync(Ls.work2 + s0, 0, sizeof(VT) * (e - s0), st));
        launch_trsv<VT, WT>(L.view, 1, L.smem_rows, nullptr, Ls.work2, nullptr, d.scratch, st);
        LevelView<VT, WT> v0 = L.view;
        v0.k = 0;
        launch_couple<VT, WT>(v0, Ls.zeros, Ls.work2, d.partial, d.counter, d.u, st);
        learned_rho_and_update<VT>(Ls, e, work, st);
        if (out_final) launch_cast_out<VT>(ntail, work + e, out_final + e, st);
    }
    for (int l = nl - 1; l >= from; --l) {
        ProfScope ps(kUp[std::min(l, 4)], st);
        launch_trsv<VT, WT>(d.lev[l].view, 1, d.lev[l].smem_rows, nullptr, work, out_final, d.scratch, st);
    }
}

template <>
void apply_hierarchy<double, double>(DevHierarchy<double, double> &d, int64_t, const double *in, double *out,
                                     cudaStream_t st) {
    apply_levels<double, double>(d, 0, in, out, nullptr, st);
}

template <>
void apply_hierarchy<float, __nv_bfloat16>(DevHierarchy<float, __nv_bfloat16> &d, int64_t, const double *in,
                                           double *out, cudaStream_t st) {
    apply_levels<float, __nv_bfloat16>(d, 0, in, d.work, out, st);
}

template void upload_hierarchy<double, double>(const Hierarchy &, Arena &, DevHierarchy<double, double> &, int);
template void upload_hierarchy<float, __nv_bfloat16>(const Hierarchy &, Arena &,
                                                     DevHierarchy<float, __nv_bfloat16> &, int);
template void upload_hierarchy<zc, zc>(const Hierarchy &, Arena &, DevHierarchy<zc, zc> &, int);
template void apply_levels<zc, zc>(DevHierarchy<zc, zc> &, int, const zc *, zc *, zc *, cudaStream_t,
                                   const PendingLowRank<zc, zc> &);
template void set_lowrank<double, double>(DevLevel<double, double> &, const HostLevel &, Arena &);
template void apply_levels<double, double>(DevHierarchy<double, double> &, int, const double *, double *, double *,
                                           cudaStream_t, const PendingLowRank<double, double> &);
template void setup_inner<double, double>(const Hierarchy &, Arena &, DevHierarchy<double, double> &, int, int);
template void setup_inner<float, __nv_bfloat16>(const Hierarchy &, Arena &, DevHierarchy<float, __nv_bfloat16> &,
                                                int, int);

}  // namespace gemslr
