// Device layout of the GeMSLR hierarchy and the application of M^{-1} (Alg. 2).
#include <algorithm>
#include <cstring>

#include "device.h"

namespace gemslr {

void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) fail(GEMSLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Arena::~Arena() {
    for (void *p : ptrs_) cudaFree(p);
}

void *Arena::alloc(size_t bytes) {
    void *p = nullptr;
    const size_t b = bytes ? (bytes + 255) & ~size_t(255) : 256;
    if (cudaMalloc(&p, b) != cudaSuccess) {
        cudaGetLastError();
        fail(GEMSLR_ERR_NOMEM, "device allocation of " + std::to_string(b) + " bytes failed");
    }
    ptrs_.push_back(p);
    total_ += b;
    return p;
}

namespace {

template <typename T> T cast_to(double v);
template <> double cast_to<double>(double v) { return v; }
template <> float cast_to<float>(double v) { return (float)v; }
template <> __nv_bfloat16 cast_to<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

template <typename VT>
struct TriHost {
    std::vector<int32_t> blk_wf{0}, wf_slot{0}, slot_row, slot_len, ent_col;
    std::vector<int64_t> wf_ent;
    std::vector<VT> ent_val;
    int maxwf = 0;
};

// Wavefront-sliced layout of a block-diagonal triangular factor.  For U the
// diagonal is moved to dinv (as 1/u_ii).
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
                if (upper && c == i) diag = T.v[p] != 0.0;
            }
            if (upper && !diag) fail(GEMSLR_ERR_ARG, "U needs a nonzero diagonal");
        }
}

template <typename VT>
void build_tri(const Csr &T, const std::vector<int64_t> &bp, bool upper, TriHost<VT> &out, std::vector<VT> *dinv) {
    validate_tri(T, bp, upper);
    if (upper) dinv->assign(T.nrows, cast_to<VT>(0.0));
    for (size_t b = 0; b + 1 < bp.size(); ++b) {
        const int64_t r0 = bp[b], r1 = bp[b + 1];
        std::vector<int32_t> lev = upper ? wavefronts_upper(T, r0, r1) : wavefronts_lower(T, r0, r1);
        int nw = 0;
        for (int32_t x : lev) nw = std::max(nw, x + 1);
        out.maxwf = std::max(out.maxwf, nw);
        std::vector<std::vector<int64_t>> rows(nw);
        for (int64_t i = r0; i < r1; ++i) rows[lev[i - r0]].push_back(i);
        auto offdiag = [&](int64_t i) {
            int64_t c = 0;
            for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p) c += (T.ci[p] != i);
            return c;
        };
        for (int w = 0; w < nw; ++w) {
            std::vector<int64_t> &R = rows[w];
            std::stable_sort(R.begin(), R.end(), [&](int64_t a, int64_t c) { return offdiag(a) > offdiag(c); });
            const int64_t cnt = (int64_t)R.size();
            int64_t maxlen = 0;
            for (int64_t i : R) maxlen = std::max(maxlen, offdiag(i));
            const int64_t base = (int64_t)out.ent_col.size();
            out.wf_ent.push_back(base);
            out.ent_col.resize(base + cnt * maxlen, 0);
            out.ent_val.resize(base + cnt * maxlen, cast_to<VT>(0.0));
            for (int64_t t = 0; t < cnt; ++t) {
                const int64_t i = R[t];
                out.slot_row.push_back((int32_t)(i - r0));
                int64_t q = 0;
                for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p) {
                    if (T.ci[p] == i) {
                        if (upper) (*dinv)[i] = cast_to<VT>(1.0 / T.v[p]);
                        continue;
                    }
                    out.ent_col[base + q * cnt + t] = (int32_t)(T.ci[p] - r0);
                    out.ent_val[base + q * cnt + t] = cast_to<VT>(T.v[p]);
                    ++q;
                }
                out.slot_len.push_back((int32_t)q);
            }
            out.wf_slot.push_back((int32_t)out.slot_row.size());
        }
        out.blk_wf.push_back((int32_t)out.wf_ent.size());
    }
    if (out.wf_ent.empty()) out.wf_ent.push_back(0);
}

template <typename VT>
TriView<VT> upload_tri(const TriHost<VT> &t, Arena &a) {
    TriView<VT> v;
    v.blk_wf = a.upload(t.blk_wf);
    v.wf_slot = a.upload(t.wf_slot);
    v.wf_ent = a.upload(t.wf_ent);
    v.slot_row = a.upload(t.slot_row);
    v.slot_len = a.upload(t.slot_len);
    v.ent_col = a.upload(t.ent_col);
    v.ent_val = a.upload(t.ent_val);
    return v;
}

template <typename T>
std::vector<T> convert(const std::vector<double> &x) {
    std::vector<T> y(x.size());
    for (size_t i = 0; i < x.size(); ++i) y[i] = cast_to<T>(x[i]);
    return y;
}

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
    d.smem_rows = (maxrows * (int64_t)sizeof(VT) <= smem_limit) ? (int)maxrows : 0;
    TriHost<VT> L, U;
    std::vector<VT> dinv;
    build_tri<VT>(hl.L, hl.bp, false, L, nullptr);
    build_tri<VT>(hl.U, hl.bp, true, U, &dinv);
    v.L = upload_tri(L, a);
    v.U = upload_tri(U, a);
    v.dinv = a.upload(dinv);
    d.nwf_L = L.maxwf;
    d.nwf_U = U.maxwf;
    d.nnz_tri = hl.L.nnz() + hl.U.nnz();
    if (schur) {
        std::vector<int32_t> fci(hl.F.ci.size());
        for (size_t p = 0; p < fci.size(); ++p) fci[p] = (int32_t)(hl.F.ci[p] + hl.e);
        v.F_rp = a.upload(hl.F.rp);
        v.F_ci = a.upload(fci);
        v.F_v = a.upload(convert<VT>(hl.F.v));
        v.E_rp = a.upload(hl.E.rp);
        v.E_ci = a.upload(hl.E.ci);
        v.E_v = a.upload(convert<VT>(hl.E.v));
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

template <typename VT, typename WT>
void upload_hierarchy(const Hierarchy &h, Arena &a, DevHierarchy<VT, WT> &d, int smem_limit) {
    set_trsv_smem_limit<VT, WT>(smem_limit);
    d.lev.resize(h.lev.size());
    int64_t maxd = 1;
    for (size_t l = 0; l < h.lev.size(); ++l) {
        upload_level<VT, WT>(h.lev[l], h.n, true, a, d.lev[l], smem_limit);
        set_lowrank<VT, WT>(d.lev[l], h.lev[l], a);
        maxd = std::max(maxd, h.lev[l].e - h.lev[l].s);
    }
    upload_level<VT, WT>(h.last, h.n, false, a, d.last, smem_limit);
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
void apply_levels(DevHierarchy<VT, WT> &d, int from, const double *in, VT *work, double *out_final,
                  cudaStream_t st) {
    const int nl = (int)d.lev.size();
    for (int l = from; l < nl; ++l) {
        DevLevel<VT, WT> &L = d.lev[l];
        const double *src = (l == from) ? in : nullptr;
        launch_trsv<VT, WT>(L.view, 0, L.smem_rows, src, work, nullptr, d.scratch, st);
        launch_couple<VT, WT>(L.view, src, work, d.partial, d.counter, d.u, st);
        launch_lowrank<VT, WT>(L.view, work, d.u, st);
    }
    launch_trsv<VT, WT>(d.last.view, 0, d.last.smem_rows, from == nl ? in : nullptr, work, out_final, d.scratch, st);
    for (int l = nl - 1; l >= from; --l)
        launch_trsv<VT, WT>(d.lev[l].view, 1, d.lev[l].smem_rows, nullptr, work, out_final, d.scratch, st);
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
template void set_lowrank<double, double>(DevLevel<double, double> &, const HostLevel &, Arena &);
template void apply_levels<double, double>(DevHierarchy<double, double> &, int, const double *, double *, double *,
                                           cudaStream_t);

}  // namespace gemslr
