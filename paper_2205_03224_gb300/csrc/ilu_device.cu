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

}  // namespace gemslr
