// The complex-shifted method (Sec. 5.2.3): every diagonal block is factored
// as B + i alpha I, so the factors, the low-rank corrections W H W^H (from the
// Arnoldi in complex arithmetic, Sec. 2.2-2.3) and every vector of M^{-1}
// and of FGMRES are complex.  M^{-1} runs the same staged substitution and
// coupling kernels as the real hierarchy, instantiated for the 16-byte
// complex scalar zc; this file holds the complex Krylov kernels (products
// with the real A, V^H w reductions, Gram-Schmidt updates, the Hessenberg
// column with complex Givens rotations, the cycle's least-squares solve),
// the complex Krylov-Schur set-up of the corrections and the FGMRES driver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>

#include "device.h"
#include "ptx.cuh"

namespace gemslr {

namespace {

constexpr int kZTile = 1024;           // rows per tile of the V^H w reduction
constexpr int kZThreads = 256;

// Per-step results of the Hessenberg kernel (device; read by the host).
struct ZCtl {
    int32_t breakdown;
    int32_t nonfinite;
    double beta;       // h_{j+1,j}
    double resid;      // |g_{j+1}|
};

__global__ void k_zgather(int64_t n, const int32_t *__restrict__ perm, const zc *__restrict__ src,
                          zc *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

__global__ void k_zscatter(int64_t n, const int32_t *__restrict__ perm, const zc *__restrict__ src,
                           zc *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}

__global__ void k_zfill(int64_t n, zc *__restrict__ x, zc v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// y = A x (b == nullptr) or y = b - A x, A real CSR, x complex; four lanes per
// row.  The trip count of the grid-stride loop is the same for every thread,
// so whole warps reach the shuffles together.
__global__ void __launch_bounds__(256) k_zspmv(int64_t n, const int64_t *__restrict__ rp,
                                               const int32_t *__restrict__ ci, const double *__restrict__ v,
                                               const zc *__restrict__ x, const zc *__restrict__ b,
                                               zc *__restrict__ y) {
    const int sub = threadIdx.x & 3;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = 0; base < 4 * n; base += nth) {
        const int64_t i = (base + tid) >> 2;
        zc acc(0.0);
        if (i < n)
            for (int64_t p = rp[i] + sub; p < rp[i + 1]; p += 4) acc += v[p] * x[ci[p]];
        acc += shfl_xor(acc, 1, 4);
        acc += shfl_xor(acc, 2, 4);
        if (i < n && sub == 0) y[i] = b ? b[i] - acc : acc;
    }
}

// out[c] = V[:, c]^H w for c < ncols and out[ncols] = (||w||^2, 0).  Every CTA
// stages tiles of w in shared memory; warp q takes the columns c = q mod 8 (and
// the norm slot) over the tile; per-CTA sums go to partials (column-major),
// and the last CTA reduces them in a fixed order (deterministic).
__global__ void __launch_bounds__(kZThreads) k_zdots(int64_t len, const zc *__restrict__ V, int64_t ldv, int ncols,
                                                     const zc *__restrict__ w, zc *__restrict__ partial,
                                                     unsigned *__restrict__ counter, zc *__restrict__ out) {
    __shared__ zc ws[kZTile];
    __shared__ zc acc[kMaxCols + 1];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = threadIdx.x; c <= ncols; c += blockDim.x) acc[c] = zc(0.0);
    for (int64_t t0 = (int64_t)blockIdx.x * kZTile; t0 < len; t0 += (int64_t)gridDim.x * kZTile) {
        const int nr = (int)min((int64_t)kZTile, len - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < kZTile; i += blockDim.x) ws[i] = i < nr ? w[t0 + i] : zc(0.0);
        __syncthreads();
        for (int c = warp; c <= ncols; c += nw) {
            zc s(0.0);
            if (c < ncols) {
                const zc *vc = V + (int64_t)c * ldv + t0;
                for (int i = lane; i < nr; i += 32) s += conj(vc[i]) * ws[i];
            } else {
                double q = 0.0;
                for (int i = lane; i < nr; i += 32) q += abs2(ws[i]);
                s = zc(q);
            }
            s = warp_sum(s);
            if (lane == 0) acc[c] += s;      // column c belongs to warp c mod nw
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c <= ncols; c += blockDim.x) partial[(int64_t)c * gridDim.x + blockIdx.x] = acc[c];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    reduce_columns<zc>(partial, (int)gridDim.x, ncols + 1, acc);
    for (int c = threadIdx.x; c <= ncols; c += blockDim.x) out[c] = acc[c];
    if (threadIdx.x == 0) *counter = 0u;
}

// w -= V[:, :ncols] h
__global__ void __launch_bounds__(256) k_zsub(int64_t len, const zc *__restrict__ V, int64_t ldv, int ncols,
                                              const zc *__restrict__ h, zc *__restrict__ w) {
    __shared__ zc hs[kMaxCols];
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = h[c];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        zc a = w[i];
        for (int c = 0; c < ncols; ++c) a -= V[(int64_t)c * ldv + i] * hs[c];
        w[i] = a;
    }
}

// v = w / sqrt(n2.re) (v = 0 when the norm is zero)
__global__ void k_zscale(int64_t len, const zc *__restrict__ w, const zc *__restrict__ n2, zc *__restrict__ v) {
    const double nn = n2->re;
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = inv * w[i];
}

// out[:, t] = V[:, :mm] Q[:, t], t < kk (thick restart and W = V Q)
__global__ void k_zrotate(int64_t len, const zc *__restrict__ V, int64_t ldv, int mm, const zc *__restrict__ Q,
                          int kk, zc *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < kk; ++t) {
            zc a(0.0);
            for (int c = 0; c < mm; ++c) a += V[(int64_t)c * ldv + i] * Q[c + (int64_t)t * mm];
            out[(int64_t)t * len + i] = a;
        }
}

// Start of a cycle: g = (||r||, 0, ...), from the norm slot n2.
__global__ void k_zcycle_start(int m, const zc *__restrict__ n2, zc *__restrict__ g) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = zc(i == 0 ? sqrt(n2->re) : 0.0);
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, the
// breakdown test h_{j+1,j} <= 1e-14 ||A z_j||, the previous rotations, the
// new complex Givens rotation [[conj(c), conj(s)], [-s, c]] with
// c = h_jj / d, s = h_{j+1,j} / d, d = sqrt(|h_jj|^2 + h_{j+1,j}^2), and
// g_{j+1} = -s g_j, g_j = conj(c) g_j.  One thread (the column is short).
__global__ void k_ztail(int j, int m, zc *__restrict__ H, zc *__restrict__ cs, zc *__restrict__ sn,
                        zc *__restrict__ g, const zc *__restrict__ h1, const zc *__restrict__ h2,
                        const zc *__restrict__ nb, ZCtl *__restrict__ ctl) {
    if (threadIdx.x != 0) return;
    zc *col = H + (int64_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    const double wn0 = sqrt(h1[j + 1].re);
    const double beta = sqrt(nb->re);
    col[j + 1] = zc(beta);
    const bool breakdown = beta <= 1e-14 * wn0;
    for (int i = 0; i < j; ++i) {
        const zc t = conj(cs[i]) * col[i] + conj(sn[i]) * col[i + 1];
        col[i + 1] = -(sn[i] * col[i]) + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double d = hypot(hypot(col[j].re, col[j].im), beta);
    zc c(1.0), s(0.0);
    if (d > 0.0) {
        c = zc(col[j].re / d, col[j].im / d);
        s = zc(beta / d);
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = zc(d);
    col[j + 1] = zc(0.0);
    g[j + 1] = -(s * g[j]);
    g[j] = conj(c) * g[j];
    ctl->beta = beta;
    ctl->breakdown = breakdown ? 1 : 0;
    const double r = hypot(g[j + 1].re, g[j + 1].im);
    ctl->resid = r;
    ctl->nonfinite = (isfinite(r) && isfinite(d)) ? 0 : 1;
}

// y = R^{-1} g[0:jd] for the rotated (upper triangular) Hessenberg matrix.
__global__ void k_zlsq(int jd, int m, const zc *__restrict__ H, const zc *__restrict__ g, zc *__restrict__ y) {
    if (threadIdx.x != 0) return;
    for (int i = jd - 1; i >= 0; --i) {
        zc s = g[i];
        for (int t = i + 1; t < jd; ++t) s -= H[i + (int64_t)t * (m + 1)] * y[t];
        const zc r = H[i + (int64_t)i * (m + 1)];
        const double den = r.re * r.re + r.im * r.im;
        y[i] = zc((s.re * r.re + s.im * r.im) / den, (s.im * r.re - s.re * r.im) / den);
    }
}

// x += Z[:, :jd] y
__global__ void k_zupdate(int64_t len, const zc *__restrict__ Z, int64_t ldz, int jd, const zc *__restrict__ y,
                          zc *__restrict__ x) {
    __shared__ zc ys[kMaxCols];
    for (int c = threadIdx.x; c < jd; c += blockDim.x) ys[c] = y[c];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        zc a = x[i];
        for (int c = 0; c < jd; ++c) a += Z[(int64_t)c * ldz + i] * ys[c];
        x[i] = a;
    }
}

int grid_of(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace

struct ZState {
    Arena *arena = nullptr;
    Hierarchy *host = nullptr;
    DevHierarchy<zc, zc> d;
    int64_t n = 0;
    const int64_t *A_rp = nullptr;
    const int32_t *A_ci = nullptr;
    const double *A_v = nullptr;
    const int32_t *perm = nullptr;
    int sms = 1;
    int red_grid = 1;
    zc *zeros = nullptr;                  // n complex zeros (G_hat operator)
    zc *partial = nullptr;                // (kMaxCols + 1) x red_grid
    unsigned *counter = nullptr;
    zc *h1 = nullptr, *h2 = nullptr, *nb = nullptr;   // kMaxCols + 1 each
    ZCtl *ctl = nullptr, *ctl_host = nullptr;
    zc *scal_host = nullptr;              // pinned: read-back of reductions
    int32_t *err_host = nullptr;          // pinned
    // FGMRES workspace (restart m_alloc)
    int m_alloc = 0;
    zc *V = nullptr, *Z = nullptr, *w = nullptr, *xh = nullptr, *bh = nullptr;
    zc *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    ~ZState() {
        if (ctl_host) cudaFreeHost(ctl_host);
        if (scal_host) cudaFreeHost(scal_host);
        if (err_host) cudaFreeHost(err_host);
    }
};

namespace {

template <typename T> T *zalloc(ZState &z, size_t count) { return (T *)z.arena->alloc(sizeof(T) * std::max<size_t>(count, 1)); }

void zdots(ZState &z, int64_t len, const zc *V, int64_t ldv, int ncols, const zc *w, zc *out, cudaStream_t st) {
    const int grid = grid_of(len, kZTile, z.red_grid);
    k_zdots<<<grid, kZThreads, 0, st>>>(len, V, ldv, ncols, w, z.partial, z.counter, out);
    count_launch();
}

void zsub(int64_t len, const zc *V, int64_t ldv, int ncols, const zc *h, zc *w, int sms, cudaStream_t st) {
    if (ncols == 0) return;
    k_zsub<<<grid_of(len, 256, 8 * sms), 256, 0, st>>>(len, V, ldv, ncols, h, w);
    count_launch();
}

void zscale(int64_t len, const zc *w, const zc *n2, zc *v, int sms, cudaStream_t st) {
    k_zscale<<<grid_of(len, 256, 8 * sms), 256, 0, st>>>(len, w, n2, v);
    count_launch();
}

void zspmv(ZState &z, const zc *x, const zc *b, zc *y, cudaStream_t st) {
    k_zspmv<<<grid_of(4 * z.n, 256, 16 * z.sms), 256, 0, st>>>(z.n, z.A_rp, z.A_ci, z.A_v, x, b, y);
    count_launch();
}

void zfill(int64_t n, zc *x, zc v, int sms, cudaStream_t st) {
    k_zfill<<<grid_of(n, 256, 8 * sms), 256, 0, st>>>(n, x, v);
    count_launch();
}

std::complex<double> read_z(ZState &z, const zc *dev, cudaStream_t st) {
    GEMSLR_CUDA(cudaMemcpyAsync(z.scal_host, dev, sizeof(zc), cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
    return {z.scal_host->re, z.scal_host->im};
}

// G_hat_l z = E_l U_l^-1 L_l^-1 F_l C_l^-1 z (length n - e_l, device).
void g_hat_z(ZState &z, int l, const zc *in, zc *out, cudaStream_t st) {
    DevHierarchy<zc, zc> &d = z.d;
    const HostLevel &hl = z.host->lev[l];
    const int64_t s = z.n - hl.e, dl = hl.e - hl.s;
    zc *X = d.work;
    GEMSLR_CUDA(cudaMemcpyAsync(X + hl.e, in, sizeof(zc) * s, cudaMemcpyDeviceToDevice, st));
    apply_levels<zc, zc>(d, l + 1, nullptr, X, nullptr, st);                // y = C_l^-1 z (tail)
    GEMSLR_CUDA(cudaMemsetAsync(X + hl.s, 0, sizeof(zc) * dl, st));
    launch_trsv<zc, zc>(d.lev[l].view, 1, d.lev[l].smem_rows, nullptr, X, nullptr, d.scratch, st);
    LevelView<zc, zc> v0 = d.lev[l].view;                                   // -(LU)^-1 F y in level rows
    v0.k = 0;
    launch_couple<zc, zc>(v0, z.zeros, X, d.partial, d.counter, d.u, st);   // tail = E (LU)^-1 F y
    GEMSLR_CUDA(cudaMemcpyAsync(out, X + hl.e, sizeof(zc) * s, cudaMemcpyDeviceToDevice, st));
}

std::vector<double> real_part(const std::vector<std::complex<double>> &x) {
    std::vector<double> r(x.size());
    for (size_t i = 0; i < x.size(); ++i) r[i] = x[i].real();
    return r;
}

std::vector<double> imag_part(const std::vector<std::complex<double>> &x) {
    std::vector<double> r(x.size());
    for (size_t i = 0; i < x.size(); ++i) r[i] = x[i].imag();
    return r;
}

// 2u - 1 from splitmix64(seed): the seeded Arnoldi start vector (real).
std::vector<double> start_vector_z(uint64_t seed, int64_t s) {
    std::vector<double> v = splitmix_uniform01(seed, s);
    for (double &x : v) x = 2.0 * x - 1.0;
    return v;
}

void store_lowrank(ZState &z, HostLevel &hl, const zc *Wd, int64_t s, int keff,
                   const std::vector<std::complex<double>> &Tk, cudaStream_t st) {
    std::vector<zc> W((size_t)s * keff);
    if (!W.empty()) GEMSLR_CUDA(cudaMemcpyAsync(W.data(), Wd, sizeof(zc) * W.size(), cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
    hl.k = keff;
    hl.W.resize(W.size());
    hl.Wi.resize(W.size());
    for (size_t i = 0; i < W.size(); ++i) { hl.W[i] = W[i].re; hl.Wi[i] = W[i].im; }
    const std::vector<std::complex<double>> Hc = correction_matrix_z(Tk, keff);
    hl.H = real_part(Hc);
    hl.Hi = imag_part(Hc);
}

// Complex thick-restart (Krylov-Schur) Arnoldi on G_hat_l: classical
// Gram-Schmidt with one forced second pass (inner products v^H w), cycle
// m = 2k, the k wanted Schur vectors kept on restart; converged when
// ||beta Q[m-1, :k]||_2 <= tol * min |theta_i|; s_l <= m: dense G_hat.
void z_build_lowrank(ZState &z, int l, const gemslr_options &opt, cudaStream_t st) {
    HostLevel &hl = z.host->lev[l];
    const int64_t s = z.n - hl.e;
    const int k = std::max(0, hl.rank_req);
    hl.k = 0;
    hl.W.clear(); hl.Wi.clear(); hl.H.clear(); hl.Hi.clear();
    if (k == 0 || s == 0) return;
    const int m = 2 * k;
    std::vector<std::complex<double>> Q, Tk, th;
    if (s <= m) {
        std::vector<std::complex<double>> G((size_t)s * s);
        std::vector<zc> e(s), col(s);
        zc *ed = zalloc<zc>(z, s), *gd = zalloc<zc>(z, s);
        for (int64_t i = 0; i < s; ++i) {
            std::fill(e.begin(), e.end(), zc(0.0));
            e[i] = zc(1.0);
            GEMSLR_CUDA(cudaMemcpyAsync(ed, e.data(), sizeof(zc) * s, cudaMemcpyHostToDevice, st));
            g_hat_z(z, l, ed, gd, st);
            GEMSLR_CUDA(cudaMemcpyAsync(col.data(), gd, sizeof(zc) * s, cudaMemcpyDeviceToHost, st));
            GEMSLR_CUDA(cudaStreamSynchronize(st));
            for (int64_t r = 0; r < s; ++r) G[r + (size_t)i * s] = {col[r].re, col[r].im};
        }
        const int keff = schur_wanted_z(G, (int)s, k, Q, Tk, th);
        std::vector<zc> Wq((size_t)s * keff);
        for (size_t i = 0; i < Wq.size(); ++i) Wq[i] = zc(Q[i].real(), Q[i].imag());
        zc *Wd = zalloc<zc>(z, Wq.size());
        GEMSLR_CUDA(cudaMemcpyAsync(Wd, Wq.data(), sizeof(zc) * Wq.size(), cudaMemcpyHostToDevice, st));
        store_lowrank(z, hl, Wd, s, keff, Tk, st);
        return;
    }
    if (m + 1 > kMaxCols) fail(GEMSLR_ERR_ARG, "rank too large for the Arnoldi workspace");
    zc *V = zalloc<zc>(z, (size_t)s * (m + 1));
    zc *W2 = zalloc<zc>(z, (size_t)s * (k + 2));
    zc *w = zalloc<zc>(z, s);
    zc *Qd = zalloc<zc>(z, (size_t)m * (k + 2));
    {
        std::vector<double> v1 = start_vector_z(1000 + (uint64_t)l, s);
        double nv = 0.0;
        for (double x : v1) nv += x * x;
        nv = std::sqrt(nv);
        std::vector<zc> v1z(s);
        for (int64_t i = 0; i < s; ++i) v1z[i] = zc(v1[i] / nv);
        GEMSLR_CUDA(cudaMemcpyAsync(V, v1z.data(), sizeof(zc) * s, cudaMemcpyHostToDevice, st));
        GEMSLR_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<std::complex<double>> Hb((size_t)(m + 1) * m, 0.0);
    std::vector<zc> hv1(kMaxCols + 1), hv2(kMaxCols + 1);
    const double tol = opt.arnoldi_tol > 0 ? opt.arnoldi_tol : 1e-2;
    const int maxc = opt.arnoldi_max_cycles > 0 ? opt.arnoldi_max_cycles : 20;
    int p = 0;
    for (int cycle = 0; cycle < maxc; ++cycle) {
        int mm = m;
        bool broke = false;
        double beta = 0.0;
        for (int j = p; j < m; ++j) {
            g_hat_z(z, l, V + (size_t)j * s, w, st);
            zdots(z, s, V, s, j + 1, w, z.h1, st);
            zsub(s, V, s, j + 1, z.h1, w, z.sms, st);
            zdots(z, s, V, s, j + 1, w, z.h2, st);
            zsub(s, V, s, j + 1, z.h2, w, z.sms, st);
            zdots(z, s, V, s, 0, w, z.nb, st);
            GEMSLR_CUDA(cudaMemcpyAsync(hv1.data(), z.h1, sizeof(zc) * (j + 2), cudaMemcpyDeviceToHost, st));
            GEMSLR_CUDA(cudaMemcpyAsync(hv2.data(), z.h2, sizeof(zc) * (j + 1), cudaMemcpyDeviceToHost, st));
            const std::complex<double> nbv = read_z(z, z.nb, st);
            const double wn0 = std::sqrt(hv1[j + 1].re);
            beta = std::sqrt(nbv.real());
            for (int i = 0; i <= j; ++i)
                Hb[i + (size_t)j * (m + 1)] = {hv1[i].re + hv2[i].re, hv1[i].im + hv2[i].im};
            Hb[(j + 1) + (size_t)j * (m + 1)] = beta;
            if (beta <= 1e-14 * std::max(wn0, 1e-300)) { mm = j + 1; broke = true; beta = 0.0; break; }
            zscale(s, w, z.nb, V + (size_t)(j + 1) * s, z.sms, st);
        }
        std::vector<std::complex<double>> Hm((size_t)mm * mm);
        for (int j = 0; j < mm; ++j)
            for (int i = 0; i < mm; ++i) Hm[i + (size_t)j * mm] = Hb[i + (size_t)j * (m + 1)];
        const int keff = schur_wanted_z(Hm, mm, k, Q, Tk, th);
        double res = 0.0, tmin = INFINITY;
        for (int t = 0; t < keff; ++t) {
            res += std::norm(beta * Q[(mm - 1) + (size_t)t * mm]);
            tmin = std::min(tmin, std::abs(th[t]));
        }
        res = std::sqrt(res);
        const bool ok = broke || res <= tol * tmin;
        std::vector<zc> Qz((size_t)mm * keff);
        for (size_t i = 0; i < Qz.size(); ++i) Qz[i] = zc(Q[i].real(), Q[i].imag());
        GEMSLR_CUDA(cudaMemcpyAsync(Qd, Qz.data(), sizeof(zc) * Qz.size(), cudaMemcpyHostToDevice, st));
        k_zrotate<<<grid_of(s, 256, 8 * z.sms), 256, 0, st>>>(s, V, s, mm, Qd, keff, W2);
        count_launch();
        if (ok || cycle == maxc - 1) {
            store_lowrank(z, hl, W2, s, keff, Tk, st);
            return;
        }
        // thick restart: V[:, :keff] = V Q, V[:, keff] = v_{m+1}
        GEMSLR_CUDA(cudaMemcpyAsync(V + (size_t)keff * s, V + (size_t)mm * s, sizeof(zc) * s,
                                    cudaMemcpyDeviceToDevice, st));
        GEMSLR_CUDA(cudaMemcpyAsync(V, W2, sizeof(zc) * (size_t)s * keff, cudaMemcpyDeviceToDevice, st));
        GEMSLR_CUDA(cudaStreamSynchronize(st));
        std::fill(Hb.begin(), Hb.end(), 0.0);
        for (int b = 0; b < keff; ++b) {
            for (int a = 0; a < keff; ++a) Hb[a + (size_t)b * (m + 1)] = Tk[a + (size_t)b * keff];
            Hb[keff + (size_t)b * (m + 1)] = beta * Q[(mm - 1) + (size_t)b * mm];
        }
        p = keff;
    }
}

void ensure_zkrylov(ZState &z, int m) {
    if (z.m_alloc >= m) return;
    const size_t n = (size_t)std::max<int64_t>(z.n, 1);
    z.V = zalloc<zc>(z, n * (m + 1));
    z.Z = zalloc<zc>(z, n * m);
    z.H = zalloc<zc>(z, (size_t)(m + 1) * m);
    z.cs = zalloc<zc>(z, m);
    z.sn = zalloc<zc>(z, m);
    z.g = zalloc<zc>(z, m + 1);
    z.y = zalloc<zc>(z, m);
    z.m_alloc = m;
}

}  // namespace

ZState *z_create(Hierarchy &h, Arena &a, const gemslr_options &opt, const int64_t *A_rp, const int32_t *A_ci,
                 const double *A_v, const int32_t *perm, int smem_limit, int sms, bool compute_lowrank) {
    std::unique_ptr<ZState> z(new ZState());
    z->arena = &a;
    z->host = &h;
    z->n = h.n;
    z->A_rp = A_rp;
    z->A_ci = A_ci;
    z->A_v = A_v;
    z->perm = perm;
    z->sms = std::max(1, sms);
    z->red_grid = 2 * z->sms;
    const size_t n = (size_t)std::max<int64_t>(h.n, 1);
    upload_hierarchy<zc, zc>(h, a, z->d, smem_limit);
    z->zeros = zalloc<zc>(*z, n);
    GEMSLR_CUDA(cudaMemset(z->zeros, 0, sizeof(zc) * n));
    z->partial = zalloc<zc>(*z, (size_t)(kMaxCols + 1) * z->red_grid);
    z->counter = zalloc<unsigned>(*z, 4);
    GEMSLR_CUDA(cudaMemset(z->counter, 0, sizeof(unsigned) * 4));
    z->h1 = zalloc<zc>(*z, kMaxCols + 1);
    z->h2 = zalloc<zc>(*z, kMaxCols + 1);
    z->nb = zalloc<zc>(*z, 1);
    z->ctl = zalloc<ZCtl>(*z, 1);
    z->w = zalloc<zc>(*z, n);
    z->xh = zalloc<zc>(*z, n);
    z->bh = zalloc<zc>(*z, n);
    GEMSLR_CUDA(cudaMallocHost(&z->ctl_host, sizeof(ZCtl)));
    GEMSLR_CUDA(cudaMallocHost(&z->scal_host, sizeof(zc)));
    GEMSLR_CUDA(cudaMallocHost(&z->err_host, sizeof(int32_t)));
    if (compute_lowrank) {
        cudaStream_t st = nullptr;
        for (int l = (int)h.lev.size() - 1; l >= 0; --l) {   // bottom-up (Sec. 4.2)
            z_build_lowrank(*z, l, opt, st);
            set_lowrank<zc, zc>(z->d.lev[l], h.lev[l], a);
        }
    }
    GEMSLR_CUDA(cudaDeviceSynchronize());
    return z.release();
}

void z_destroy(ZState *z) { delete z; }

void z_wavefronts(const ZState *z, int l, int &wl, int &wu) {
    const DevLevel<zc, zc> &d = l < (int)z->d.lev.size() ? z->d.lev[l] : z->d.last;
    wl = d.nwf_L;
    wu = d.nwf_U;
}

void z_apply(ZState *z, const zc *r, zc *out, int32_t nrhs, cudaStream_t st) {
    const int64_t n = z->n;
    for (int c = 0; c < nrhs; ++c) {
        k_zgather<<<grid_of(n, 256, 8 * z->sms), 256, 0, st>>>(n, z->perm, r + (size_t)c * n, z->bh);
        count_launch();
        apply_levels<zc, zc>(z->d, 0, z->bh, z->xh, nullptr, st);
        k_zscatter<<<grid_of(n, 256, 8 * z->sms), 256, 0, st>>>(n, z->perm, z->xh, out + (size_t)c * n);
        count_launch();
    }
    GEMSLR_CUDA(cudaGetLastError());
}

// Restarted FGMRES(m) in complex arithmetic for one right-hand side (Sec. 4.1).
gemslr_status z_solve(ZState *zp, const zc *b, zc *x, const gemslr_solve_opts &o, gemslr_solve_info &inf,
                      std::string &msg, cudaStream_t st) {
    ZState &z = *zp;
    const int64_t n = z.n;
    const int m = o.restart;
    if (m + 1 > kMaxCols) fail(GEMSLR_ERR_ARG, "restart too large (m + 1 <= 160)");
    ensure_zkrylov(z, m);
    auto t0 = std::chrono::steady_clock::now();
    std::memset(&inf, 0, sizeof(inf));
    const int gs = grid_of(n, 256, 8 * z.sms);
    k_zgather<<<gs, 256, 0, st>>>(n, z.perm, b, z.bh);
    count_launch();
    zfill(n, z.xh, zc(0.0), z.sms, st);
    zdots(z, n, nullptr, n, 0, z.bh, z.nb, st);
    const double bnorm = std::sqrt(read_z(z, z.nb, st).real());
    gemslr_status status = GEMSLR_OK;
    if (!std::isfinite(bnorm) || bnorm == 0.0) {
        k_zscatter<<<gs, 256, 0, st>>>(n, z.perm, z.xh, x);
        count_launch();
        GEMSLR_CUDA(cudaStreamSynchronize(st));
        if (bnorm == 0.0) {
            inf.converged = 1;
            return GEMSLR_OK;
        }
        msg = "right-hand side is not finite";
        return GEMSLR_ERR_NAN;
    }
    const double tol = o.rtol * bnorm;
    int its = 0, restarts = 0;
    bool converged = false, nonfinite = false;
    double rnorm = bnorm, resid = bnorm;
    // r_0 = b (x_0 = 0): V[:, 0] = b / ||b||
    zscale(n, z.bh, z.nb, z.V, z.sms, st);
    while (!converged && its < o.maxit) {
        k_zcycle_start<<<1, 256, 0, st>>>(m, z.nb, z.g);
        count_launch();
        int jd = 0;
        for (int j = 0; j < m; ++j) {
            zc *vj = z.V + (size_t)j * n, *zj = z.Z + (size_t)j * n;
            apply_levels<zc, zc>(z.d, 0, vj, zj, nullptr, st);      // z_j = M^{-1} v_j
            zspmv(z, zj, nullptr, z.w, st);                        // w = A z_j
            zdots(z, n, z.V, n, j + 1, z.w, z.h1, st);            // classical Gram-Schmidt, two passes
            zsub(n, z.V, n, j + 1, z.h1, z.w, z.sms, st);
            zdots(z, n, z.V, n, j + 1, z.w, z.h2, st);
            zsub(n, z.V, n, j + 1, z.h2, z.w, z.sms, st);
            zdots(z, n, nullptr, n, 0, z.w, z.nb, st);
            k_ztail<<<1, 32, 0, st>>>(j, m, z.H, z.cs, z.sn, z.g, z.h1, z.h2, z.nb, z.ctl);
            count_launch();
            zscale(n, z.w, z.nb, z.V + (size_t)(j + 1) * n, z.sms, st);
            GEMSLR_CUDA(cudaMemcpyAsync(z.ctl_host, z.ctl, sizeof(ZCtl), cudaMemcpyDeviceToHost, st));
            GEMSLR_CUDA(cudaStreamSynchronize(st));
            ++its;
            jd = j + 1;
            resid = z.ctl_host->resid;
            if (z.ctl_host->nonfinite) { nonfinite = true; break; }
            if (resid <= tol || z.ctl_host->breakdown || its >= o.maxit) break;
        }
        if (nonfinite) break;
        k_zlsq<<<1, 32, 0, st>>>(jd, m, z.H, z.g, z.y);
        k_zupdate<<<gs, 256, 0, st>>>(n, z.Z, n, jd, z.y, z.xh);
        count_launch(2);
        zspmv(z, z.xh, z.bh, z.w, st);                              // r = b - A x
        zdots(z, n, nullptr, n, 0, z.w, z.nb, st);
        rnorm = std::sqrt(read_z(z, z.nb, st).real());
        if (!std::isfinite(rnorm)) { nonfinite = true; break; }
        converged = rnorm <= tol;
        if (!converged) {
            ++restarts;
            zscale(n, z.w, z.nb, z.V, z.sms, st);
        }
    }
    k_zscatter<<<gs, 256, 0, st>>>(n, z.perm, z.xh, x);
    count_launch();
    GEMSLR_CUDA(cudaMemcpyAsync(z.err_host, z.d.err, 4, cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
    inf.iters = its;
    inf.restarts = restarts;
    inf.converged = converged ? 1 : 0;
    inf.reorth = its;
    inf.rel_res_est = resid / bnorm;
    inf.rel_res_true = rnorm / bnorm;
    inf.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (z.err_host[0]) {
        GEMSLR_CUDA(cudaMemsetAsync(z.d.err, 0, 4, st));
        fail(GEMSLR_ERR_TIMEOUT, "a bounded wait in the substitution kernel expired");
    }
    if (nonfinite) {
        msg = "FGMRES produced a non-finite value";
        status = GEMSLR_ERR_NAN;
    } else if (!converged) {
        msg = "FGMRES reached maxit";
        status = GEMSLR_ERR_NOT_CONVERGED;
    }
    return status;
}

}  // namespace gemslr
