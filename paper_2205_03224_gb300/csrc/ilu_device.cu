// ILU(0) of the diagonal blocks of one level on the GPU (set-up, Alg. 1
// "Compute ILU factorization"), level-scheduled: one CTA per diagonal block
// (the blocks are independent, Sec. 4.2) walks the block's wavefronts of the
// lower pattern in order, one thread per row of a wavefront.  Row i is
// eliminated in place in the IKJ form restricted to the pattern of B, with
// the same operations in the same order as the host factorisation (products
// and differences rounded separately, IEEE division and square root), so the
// factors are bit-identical to the host ILU(0).
#include <algorithm>
#include <cmath>
#include <vector>

#include "device.h"

namespace gemslr {

namespace {

constexpr int kIluThreads = 256;

__global__ void __launch_bounds__(kIluThreads)
k_ilu0_blocks(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, double *__restrict__ v,
              const int64_t *__restrict__ dptr, const int32_t *__restrict__ order, const int32_t *__restrict__ wf_ptr,
              const int32_t *__restrict__ blk_wf, unsigned long long *__restrict__ nclamp) {
    const int b = blockIdx.x;
    for (int w = blk_wf[b]; w < blk_wf[b + 1]; ++w) {
        for (int t = wf_ptr[w] + threadIdx.x; t < wf_ptr[w + 1]; t += blockDim.x) {
            const int64_t i = order[t];
            const int64_t p0 = rp[i], p1 = rp[i + 1], di = dptr[i];
            double nrm2 = 0.0;                          // ||a_i||_2 of the original row
            for (int64_t p = p0; p < p1; ++p) nrm2 = __dadd_rn(nrm2, __dmul_rn(v[p], v[p]));
            const double nrm = sqrt(nrm2);
            for (int64_t p = p0; p < di; ++p) {         // multipliers in ascending column order
                const int64_t k = ci[p];
                const double lik = v[p] / v[dptr[k]];
                v[p] = lik;
                int64_t r = p + 1;                      // row i's columns ascend: search forward
                for (int64_t q = dptr[k] + 1; q < rp[k + 1]; ++q) {
                    const int32_t j = ci[q];
                    while (r < p1 && ci[r] < j) ++r;
                    if (r < p1 && ci[r] == j) v[r] = __dsub_rn(v[r], __dmul_rn(lik, v[q]));
                }
            }
            double d = v[di];                           // small pivots as on the host
            if (nrm == 0.0) {
                if (d == 0.0) { d = 1.0; atomicAdd(nclamp, 1ull); }
            } else {
                const double floor_ = 1e-12 * nrm;
                if (fabs(d) < floor_) { d = d < 0.0 ? -floor_ : floor_; atomicAdd(nclamp, 1ull); }
            }
            v[di] = d;
        }
        __syncthreads();                                // the wavefront's rows before the next one's reads
    }
}

// ---- ILUT(tau, lfil) on the GPU --------------------------------------------------
// The rows of a block depend on one another through fill that only the values
// decide, so a block's rows are factored in order, one warp per block (the
// blocks are independent).  The row's values live in a dense work array of
// the level (global memory, indexed by column); its column list, elimination
// flags and candidates live in shared memory: the smallest not-yet-eliminated
// column below the diagonal is a warp minimum over the list, it is eliminated
// with the finished U row (new fill columns appended by a warp ballot), and the
// lfil largest L and U candidates are picked by warp arg-max rounds over the
// candidates gathered once (ties: lower column), then sorted by column.
// Every operation and its order follow the host ILUT (products, differences,
// divisions and the square root rounded separately), so the factors are
// bit-identical to it.  A row touching more than kIlutSlots columns sets the
// overflow word, and the host factors that level itself.
constexpr int kIlutWarps = 4;
constexpr int kMaxIlutFill = 64;           // lfil bound of the device ILUT
constexpr int kIlutSlots = 512;            // columns of one row held in shared memory

struct IlutWork {
    double *row;               // n, dense work row (level-local columns), zero between rows
    double *piv;               // n, guarded pivots u_ii
    unsigned char *present;    // n
    int32_t *Lc, *Uc;          // n x capL, n x capU
    double *Lv, *Uv;
    int32_t *Ln, *Un;          // n
    int32_t *overflow;         // set when a row has more than kIlutSlots columns
};

__device__ __forceinline__ bool better(double ma, int ca, double mb, int cb) {
    return ma > mb || (ma == mb && ca < cb);
}

// The lfil largest candidates (lower: c < i, |row_c piv_c| >= thr; upper:
// c > i, |row_c| >= thr; row_c != 0) of the row, sorted by column into list.
__device__ int ilut_select(const IlutWork &W, const int32_t *scol, int ncols, int64_t i, bool lower, double thr,
                           int lfil, int32_t *ccol, double *cmag, int32_t *list, int lane) {
    int m = 0;                                   // candidates, gathered once into shared memory
    for (int t0 = 0; t0 < ncols; t0 += 32) {
        const int t = t0 + lane;
        bool ok = false;
        double mag = 0.0;
        int c = 0;
        if (t < ncols) {
            c = scol[t];
            const double r = W.row[c];
            if ((lower ? (int64_t)c < i : (int64_t)c > i) && r != 0.0) {
                mag = fabs(lower ? __dmul_rn(r, W.piv[c]) : r);
                ok = mag >= thr;
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int pos = m + __popc(mask & ((1u << lane) - 1u));
            ccol[pos] = c;
            cmag[pos] = mag;
        }
        m += __popc(mask);
    }
    __syncwarp();
    if (m > lfil) {                       // keep the lfil largest (ties: lower column)
        for (int r = 0; r < lfil; ++r) {
            double bm = -1.0;
            int bc = 0x7fffffff, bt = -1;
            for (int t = lane; t < m; t += 32)
                if (cmag[t] >= 0.0 && better(cmag[t], ccol[t], bm, bc)) { bm = cmag[t]; bc = ccol[t]; bt = t; }
            for (int o = 16; o > 0; o >>= 1) {
                const double om = __shfl_xor_sync(0xffffffffu, bm, o);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
                const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
                if (better(om, oc, bm, bc)) { bm = om; bc = oc; bt = ot; }
            }
            if (lane == 0) { list[r] = bc; cmag[bt] = -1.0; }
            __syncwarp();
        }
        m = lfil;
    } else {
        for (int t = lane; t < m; t += 32) list[t] = ccol[t];
        __syncwarp();
    }
    if (lane == 0)                        // ascending columns (m <= lfil <= kMaxIlutFill)
        for (int a = 1; a < m; ++a) {
            const int v = list[a];
            int b = a - 1;
            while (b >= 0 && list[b] > v) { list[b + 1] = list[b]; --b; }
            list[b + 1] = v;
        }
    __syncwarp();
    return m;
}

__global__ void __launch_bounds__(32 * kIlutWarps)
k_ilut_blocks(int nblk, const int64_t *__restrict__ bp, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
              const double *__restrict__ v, double tau, int lfil, IlutWork W, unsigned long long *nclamp) {
    __shared__ int32_t s_col[kIlutWarps][kIlutSlots];
    __shared__ int32_t s_ccol[kIlutWarps][kIlutSlots];
    __shared__ double s_cmag[kIlutWarps][kIlutSlots];
    __shared__ unsigned char s_elim[kIlutWarps][kIlutSlots];
    __shared__ int32_t lists[kIlutWarps][kMaxIlutFill];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kIlutWarps + warp;
    if (b >= nblk) return;
    const int capL = lfil, capU = lfil + 1;
    int32_t *list = lists[warp], *scol = s_col[warp];
    unsigned char *selim = s_elim[warp];
    const int64_t r0 = bp[b], r1 = bp[b + 1];
    for (int64_t i = r0; i < r1; ++i) {
        const int64_t p0 = rp[i], p1 = rp[i + 1];
        int ncols = (int)(p1 - p0);
        if (ncols > kIlutSlots) {                   // the warp stops; the host factors the level
            if (lane == 0) atomicExch(W.overflow, 1);
            return;
        }
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int c = ci[p];
            W.row[c] = v[p];
            W.present[c] = 1;
            scol[p - p0] = c;
            selim[p - p0] = 0;
        }
        double nrm2 = 0.0;                          // ||a_i||_2 in the row's order
        if (lane == 0)
            for (int64_t p = p0; p < p1; ++p) nrm2 = __dadd_rn(nrm2, __dmul_rn(v[p], v[p]));
        const double nrm = __shfl_sync(0xffffffffu, __dsqrt_rn(nrm2), 0);
        const double thr = __dmul_rn(tau, nrm);
        __syncwarp();
        bool over = false;
        while (true) {                              // smallest not-yet-eliminated column below the diagonal
            int k = 0x7fffffff, kt = -1;
            for (int t = lane; t < ncols; t += 32) {
                const int c = scol[t];
                if ((int64_t)c < i && !selim[t] && c < k) { k = c; kt = t; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const int ok = __shfl_xor_sync(0xffffffffu, k, o), ot = __shfl_xor_sync(0xffffffffu, kt, o);
                if (ok < k) { k = ok; kt = ot; }
            }
            if (k == 0x7fffffff) break;
            const double rk = W.row[k];
            __syncwarp();
            if (lane == 0) selim[kt] = 1;
            if (fabs(rk) < thr) {
                if (lane == 0) W.row[k] = 0.0;
                __syncwarp();
                continue;
            }
            const double lik = __ddiv_rn(rk, W.piv[k]);
            if (lane == 0) W.row[k] = lik;
            const int nu = W.Un[k];
            for (int q0 = 1; q0 < nu; q0 += 32) {   // U row k without its diagonal (first)
                const int q = q0 + lane;
                bool fresh = false;
                int j = 0;
                if (q < nu) {
                    j = W.Uc[(int64_t)k * capU + q];
                    const double u = W.Uv[(int64_t)k * capU + q];
                    fresh = !W.present[j];
                    const double rj = fresh ? 0.0 : W.row[j];
                    if (fresh) W.present[j] = 1;
                    W.row[j] = __dsub_rn(rj, __dmul_rn(lik, u));
                }
                const unsigned mask = __ballot_sync(0xffffffffu, fresh);
                const int pos = ncols + __popc(mask & ((1u << lane) - 1u));
                if (fresh && pos < kIlutSlots) {
                    scol[pos] = j;
                    selim[pos] = 0;
                }
                ncols += __popc(mask);
            }
            if (ncols > kIlutSlots) {               // too wide: the host factors this level
                over = true;
                ncols = kIlutSlots;
                break;
            }
            __syncwarp();
        }
        if (over) {
            __syncwarp();
            if (lane == 0) atomicExch(W.overflow, 1);
            return;
        }
        const int nl = ilut_select(W, scol, ncols, i, true, thr, lfil, s_ccol[warp], s_cmag[warp], list, lane);
        for (int t = lane; t < nl; t += 32) {
            W.Lc[i * capL + t] = list[t];
            W.Lv[i * capL + t] = W.row[list[t]];
        }
        if (lane == 0) {                            // the pivot, guarded as on the host
            double d = W.present[i] ? W.row[i] : 0.0;
            if (nrm == 0.0) {
                if (d == 0.0) { d = 1.0; atomicAdd(nclamp, 1ull); }
            } else {
                const double floor_ = __dmul_rn(1e-12, nrm);
                if (fabs(d) < floor_) { d = d < 0.0 ? -floor_ : floor_; atomicAdd(nclamp, 1ull); }
            }
            W.piv[i] = d;
            W.Ln[i] = nl;
            W.Uc[i * capU] = (int32_t)i;
            W.Uv[i * capU] = d;
        }
        __syncwarp();
        const int nuu = ilut_select(W, scol, ncols, i, false, thr, lfil, s_ccol[warp], s_cmag[warp], list, lane);
        for (int t = lane; t < nuu; t += 32) {
            W.Uc[i * capU + 1 + t] = list[t];
            W.Uv[i * capU + 1 + t] = W.row[list[t]];
        }
        if (lane == 0) W.Un[i] = 1 + nuu;
        __syncwarp();
        for (int t = lane; t < ncols; t += 32) {    // clean the dense work arrays for the next row
            const int c = scol[t];
            W.row[c] = 0.0;
            W.present[c] = 0;
        }
        __syncwarp();
    }
}

template <typename T>
T *dev_upload(const std::vector<T> &h, std::vector<void *> &owned) {
    void *p = nullptr;
    GEMSLR_CUDA(cudaMalloc(&p, std::max<size_t>(1, h.size()) * sizeof(T)));
    owned.push_back(p);
    if (!h.empty()) GEMSLR_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return static_cast<T *>(p);
}

}  // namespace

// L (strictly lower) and U (diagonal first) of every diagonal block of the
// level matrix B (level-local, blocks bp), factored on the current device.
// Every row needs its diagonal entry.  Temporary device buffers only.
void factor_level_ilu0_device(const Csr &B, const std::vector<int64_t> &bp, Csr &L, Csr &U, int64_t &clamped) {
    const int64_t n = B.nrows;
    std::vector<int64_t> dptr(n, -1);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
            if (B.ci[p] == i) dptr[i] = p;
    for (int64_t i = 0; i < n; ++i)
        if (dptr[i] < 0) fail(GEMSLR_ERR_ARG, "device ILU(0) needs every diagonal entry in the pattern");
    // wavefronts of the lower pattern, per block
    std::vector<int32_t> lev(n, 0), order, wf_ptr{0}, blk_wf{0};
    for (size_t b = 0; b + 1 < bp.size(); ++b) {
        int32_t nw = 0;
        for (int64_t i = bp[b]; i < bp[b + 1]; ++i) {
            int32_t m = 0;
            for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
                if (B.ci[p] < i) {
                    if (B.ci[p] < bp[b]) fail(GEMSLR_ERR_PARTITION, "a diagonal block is coupled to another");
                    m = std::max(m, lev[B.ci[p]] + 1);
                }
            lev[i] = m;
            nw = std::max(nw, m + 1);
        }
        std::vector<std::vector<int32_t>> rows(nw);
        for (int64_t i = bp[b]; i < bp[b + 1]; ++i) rows[lev[i]].push_back((int32_t)i);
        for (auto &r : rows) {
            order.insert(order.end(), r.begin(), r.end());
            wf_ptr.push_back((int32_t)order.size());
        }
        blk_wf.push_back((int32_t)wf_ptr.size() - 1);
    }
    std::vector<void *> owned;
    try {
        int64_t *d_rp = dev_upload(B.rp, owned);
        int32_t *d_ci = dev_upload(B.ci, owned);
        double *d_v = dev_upload(B.v, owned);
        int64_t *d_dp = dev_upload(dptr, owned);
        int32_t *d_or = dev_upload(order, owned);
        int32_t *d_wf = dev_upload(wf_ptr, owned);
        int32_t *d_bw = dev_upload(blk_wf, owned);
        std::vector<unsigned long long> zero(1, 0ull);
        unsigned long long *d_cl = dev_upload(zero, owned);
        const int nb = (int)bp.size() - 1;
        if (nb > 0) k_ilu0_blocks<<<nb, kIluThreads>>>(d_rp, d_ci, d_v, d_dp, d_or, d_wf, d_bw, d_cl);
        GEMSLR_CUDA(cudaGetLastError());
        std::vector<double> val(B.v.size());
        if (!val.empty()) GEMSLR_CUDA(cudaMemcpy(val.data(), d_v, val.size() * sizeof(double), cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(zero.data(), d_cl, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        clamped += (int64_t)zero[0];
        L.nrows = L.ncols = U.nrows = U.ncols = n;
        L.rp.assign(1, 0);
        U.rp.assign(1, 0);
        L.ci.clear(); L.v.clear(); U.ci.clear(); U.v.clear();
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
                if (B.ci[p] < i) { L.ci.push_back(B.ci[p]); L.v.push_back(val[p]); }
            U.ci.push_back((int32_t)i);
            U.v.push_back(val[dptr[i]]);
            for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
                if (B.ci[p] > i) { U.ci.push_back(B.ci[p]); U.v.push_back(val[p]); }
            L.rp.push_back((int64_t)L.ci.size());
            U.rp.push_back((int64_t)U.ci.size());
        }
    } catch (...) {
        for (void *p : owned) cudaFree(p);
        throw;
    }
    for (void *p : owned) GEMSLR_CUDA(cudaFree(p));
}

// ILUT(tau, lfil) of every diagonal block of the level matrix B on the current
// device (0 <= lfil <= 64); the same factors as the host ILUT, bit for bit.
// Returns false (nothing written) when a row touched more columns than the
// kernel holds in shared memory; the caller then factors the level on the host.
bool factor_level_ilut_device(const Csr &B, const std::vector<int64_t> &bp, double tau, int lfil, Csr &L, Csr &U,
                              int64_t &clamped) {
    if (lfil < 0 || lfil > kMaxIlutFill) fail(GEMSLR_ERR_ARG, "device ILUT needs 0 <= lfil <= 64");
    const int64_t n = B.nrows;
    for (size_t b = 0; b + 1 < bp.size(); ++b)
        for (int64_t i = bp[b]; i < bp[b + 1]; ++i)
            for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p)
                if (B.ci[p] < bp[b] || B.ci[p] >= bp[b + 1]) fail(GEMSLR_ERR_PARTITION, "a diagonal block is coupled to another");
    const int capL = lfil, capU = lfil + 1;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    std::vector<void *> owned;
    auto zeros = [&](size_t bytes) {
        void *p = nullptr;
        GEMSLR_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
        owned.push_back(p);
        GEMSLR_CUDA(cudaMemset(p, 0, std::max<size_t>(bytes, 16)));
        return p;
    };
    try {
        int64_t *d_rp = dev_upload(B.rp, owned);
        int32_t *d_ci = dev_upload(B.ci, owned);
        double *d_v = dev_upload(B.v, owned);
        int64_t *d_bp = dev_upload(bp, owned);
        IlutWork W;
        W.row = (double *)zeros(8 * nn);
        W.piv = (double *)zeros(8 * nn);
        W.present = (unsigned char *)zeros(nn);
        W.overflow = (int32_t *)zeros(4);
        W.Lc = (int32_t *)zeros(4 * nn * std::max(capL, 1));
        W.Lv = (double *)zeros(8 * nn * std::max(capL, 1));
        W.Uc = (int32_t *)zeros(4 * nn * capU);
        W.Uv = (double *)zeros(8 * nn * capU);
        W.Ln = (int32_t *)zeros(4 * nn);
        W.Un = (int32_t *)zeros(4 * nn);
        unsigned long long *d_cl = (unsigned long long *)zeros(8);
        const int nb = (int)bp.size() - 1;
        if (nb > 0)
            k_ilut_blocks<<<(nb + kIlutWarps - 1) / kIlutWarps, 32 * kIlutWarps>>>(nb, d_bp, d_rp, d_ci, d_v, tau,
                                                                                   lfil, W, d_cl);
        GEMSLR_CUDA(cudaGetLastError());
        int32_t over = 0;
        GEMSLR_CUDA(cudaMemcpy(&over, W.overflow, 4, cudaMemcpyDeviceToHost));
        if (over) {
            for (void *p : owned) GEMSLR_CUDA(cudaFree(p));
            return false;
        }
        std::vector<int32_t> Lc(nn * std::max(capL, 1)), Uc(nn * capU), Ln(nn), Un(nn);
        std::vector<double> Lv(Lc.size()), Uv(Uc.size());
        unsigned long long cl = 0;
        GEMSLR_CUDA(cudaMemcpy(Lc.data(), W.Lc, 4 * Lc.size(), cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(Lv.data(), W.Lv, 8 * Lv.size(), cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(Uc.data(), W.Uc, 4 * Uc.size(), cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(Uv.data(), W.Uv, 8 * Uv.size(), cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(Ln.data(), W.Ln, 4 * nn, cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(Un.data(), W.Un, 4 * nn, cudaMemcpyDeviceToHost));
        GEMSLR_CUDA(cudaMemcpy(&cl, d_cl, 8, cudaMemcpyDeviceToHost));
        clamped += (int64_t)cl;
        L.nrows = L.ncols = U.nrows = U.ncols = n;
        L.rp.assign(1, 0);
        U.rp.assign(1, 0);
        L.ci.clear(); L.v.clear(); L.vi.clear(); U.ci.clear(); U.v.clear(); U.vi.clear();
        for (int64_t i = 0; i < n; ++i) {
            for (int t = 0; t < Ln[i]; ++t) {
                L.ci.push_back(Lc[(size_t)i * capL + t]);
                L.v.push_back(Lv[(size_t)i * capL + t]);
            }
            for (int t = 0; t < Un[i]; ++t) {
                U.ci.push_back(Uc[(size_t)i * capU + t]);
                U.v.push_back(Uv[(size_t)i * capU + t]);
            }
            L.rp.push_back((int64_t)L.ci.size());
            U.rp.push_back((int64_t)U.ci.size());
        }
    } catch (...) {
        for (void *p : owned) cudaFree(p);
        throw;
    }
    for (void *p : owned) GEMSLR_CUDA(cudaFree(p));
    return true;
}

}  // namespace gemslr
