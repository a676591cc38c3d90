// GeMSLR handle, low-rank setup (Alg. 1 / Sec. 2.3), FGMRES (Sec. 4.1) and the C ABI.
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <unordered_map>

#include "device.h"

using namespace gemslr;

// Learned interface correction state of a handle (network and in-apply buffers).
struct LearnedHost {
    NetDev net;
    LearnedStage<double> st64;
    LearnedStage<float> st32;
    int lstar = -1;
    int64_t e = 0;
};

struct gemslr_ctx {
    int dev = -1;                  // CUDA device the handle was set up on
    Hierarchy host;
    gemslr_options opt{};
    Arena arena;
    DevHierarchy<double, double> d64;
    DevHierarchy<float, __nv_bfloat16> d32;
    bool mixed = false;
    // permuted A for the Krylov products
    int64_t *A_rp = nullptr;
    int32_t *A_ci = nullptr;
    double *A_v = nullptr;
    int spmv_lanes = 8;
    int32_t *perm = nullptr;
    double *zeros = nullptr;       // n zeros (Arnoldi operator)
    // Krylov workspace
    int m_alloc = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *xh = nullptr, *bh = nullptr, *r = nullptr;
    double *Hs = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *h2 = nullptr;
    // delayed reorthogonalisation (linear M^{-1}): unrotated H, R, per-step vectors
    double *Hraw = nullptr, *Rz = nullptr, *da = nullptr, *dcoef = nullptr, *dhprev = nullptr, *dapre = nullptr;
    double *partial2 = nullptr;          // partials of the kernel beside M^{-1}
    unsigned *counter2 = nullptr;
    double *partial = nullptr, *n2 = nullptr;
    unsigned *counter = nullptr;
    KrylovCtl *ctl = nullptr;
    KrylovCtl *ctl_host = nullptr;      // pinned
    double *n2_host = nullptr;          // pinned
    int red_grid = 0;
    double *vin = nullptr, *zout = nullptr;   // fixed in/out of M^{-1} inside the FGMRES step
    int32_t *err_host = nullptr;              // pinned copy of the substitution error word
    double setup_ms = 0.0;
    // second stream of the delayed reorthogonalisation (k_dgs_fix beside M^{-1})
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr;
    // CUDA graph of a whole FGMRES solve (conditional WHILE nodes for the cycle and step loops)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_m = 0;
    bool graph_dcgs = false;       // which step the captured graph runs
    bool graph_failed = false;
    uint64_t graph_k_top = 0, graph_k_cycle = 0, graph_k_step = 0;
    LearnedHost *learned = nullptr;
    ZState *z = nullptr;           // complex hierarchy and its Krylov workspace (complex shift)
    ~gemslr_ctx() {
        delete learned;
        z_destroy(z);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (aux_stream) cudaStreamDestroy(aux_stream);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_fork2) cudaEventDestroy(ev_fork2);
        if (ev_join2) cudaEventDestroy(ev_join2);
        if (ctl_host) cudaFreeHost(ctl_host);
        if (n2_host) cudaFreeHost(n2_host);
        if (err_host) cudaFreeHost(err_host);
    }
};

// The handle's device memory belongs to the device it was set up on: a call
// made while another device is current is an argument error, not a fault.
static void require_device(const gemslr_ctx *h) {
    int dev = -1;
    GEMSLR_CUDA(cudaGetDevice(&dev));
    if (dev != h->dev)
        fail(GEMSLR_ERR_ARG, "the handle lives on device " + std::to_string(h->dev) + " but device " +
                                 std::to_string(dev) + " is current");
}

// The real entry points refuse a complex handle and the complex ones a real one.
static void require_real(const gemslr_ctx *h) {
    if (h->host.cplx) fail(GEMSLR_ERR_ARG, "complex handle (complex shift): use gemslr_zapply / gemslr_zfgmres_solve");
}

namespace {

thread_local std::string g_last_error;

gemslr_status guard(const std::function<void()> &fn);

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int smem_optin() {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return b;
}

void ensure_krylov(gemslr_ctx *h, int m) {
    const int64_t n = std::max<int64_t>(h->host.n, 1);
    if (!h->ctl) {
        h->xh = (double *)h->arena.alloc(8 * n);
        h->bh = (double *)h->arena.alloc(8 * n);
        h->r = (double *)h->arena.alloc(8 * n);
        h->w = (double *)h->arena.alloc(8 * n);
        h->red_grid = sm_count();                 // one CTA per SM: few partials for the finisher
        h->partial = (double *)h->arena.alloc(8 * (size_t)h->red_grid * (2 * kMaxCols + 4));
        h->counter = (unsigned *)h->arena.alloc(16);
        GEMSLR_CUDA(cudaMemset(h->counter, 0, 16));
        h->n2 = (double *)h->arena.alloc(8 * 4);
        h->ctl = (KrylovCtl *)h->arena.alloc(sizeof(KrylovCtl));
        h->h2 = (double *)h->arena.alloc(8 * kMaxCols);
        h->da = (double *)h->arena.alloc(8 * kMaxCols);
        h->dcoef = (double *)h->arena.alloc(8 * kMaxCols);
        h->dhprev = (double *)h->arena.alloc(8 * kMaxCols);
        h->dapre = (double *)h->arena.alloc(8 * kMaxCols);
        h->partial2 = (double *)h->arena.alloc(8 * (size_t)h->red_grid * (kMaxCols + 2));
        h->counter2 = (unsigned *)h->arena.alloc(16);
        GEMSLR_CUDA(cudaMemset(h->counter2, 0, 16));
        h->vin = (double *)h->arena.alloc(8 * n);
        h->zout = (double *)h->arena.alloc(8 * n);
        prepare_krylov_kernels();
        GEMSLR_CUDA(cudaMallocHost(&h->ctl_host, sizeof(KrylovCtl)));
        GEMSLR_CUDA(cudaMallocHost(&h->n2_host, 8 * 4));
        GEMSLR_CUDA(cudaMallocHost(&h->err_host, 16));
    }
    if (m > h->m_alloc) {
        if (m + 1 > kMaxCols) fail(GEMSLR_ERR_ARG, "restart length too large");
        h->V = (double *)h->arena.alloc(8 * (size_t)n * (m + 1));
        h->Z = (double *)h->arena.alloc(8 * (size_t)n * m);
        h->Hs = (double *)h->arena.alloc(8 * (size_t)(m + 1) * m);
        h->cs = (double *)h->arena.alloc(8 * (size_t)(m + 1));
        h->sn = (double *)h->arena.alloc(8 * (size_t)(m + 1));
        h->g = (double *)h->arena.alloc(8 * (size_t)(m + 2));
        h->y = (double *)h->arena.alloc(8 * (size_t)(m + 1));
        h->Hraw = (double *)h->arena.alloc(8 * (size_t)(m + 1) * m);
        h->Rz = (double *)h->arena.alloc(8 * (size_t)(m + 1) * (m + 1));
        h->m_alloc = m;
    }
}

// M^{-1} on a multilevel-ordered FP64 vector (device).
void apply_perm(gemslr_ctx *h, const double *in, double *out, cudaStream_t st) {
    if (h->mixed) apply_hierarchy<float, __nv_bfloat16>(h->d32, h->host.n, in, out, st);
    else apply_hierarchy<double, double>(h->d64, h->host.n, in, out, st);
}

// G_hat_l z = E_l U_l^-1 L_l^-1 F_l C_l^-1 z for z of length n - e_l (device, FP64 hierarchy).
void g_hat(gemslr_ctx *h, int l, const double *z, double *out, cudaStream_t st) {
    DevHierarchy<double, double> &d = h->d64;
    const HostLevel &hl = h->host.lev[l];
    const int64_t s = h->host.n - hl.e, dl = hl.e - hl.s;
    double *X = d.work;
    GEMSLR_CUDA(cudaMemcpyAsync(X + hl.e, z, 8 * s, cudaMemcpyDeviceToDevice, st));
    apply_levels<double, double>(d, l + 1, nullptr, X, nullptr, st);         // y = C_l^-1 z (tail)
    GEMSLR_CUDA(cudaMemsetAsync(X + hl.s, 0, 8 * dl, st));
    launch_trsv<double, double>(d.lev[l].view, 1, d.lev[l].smem_rows, nullptr, X, nullptr, d.scratch, st);
    LevelView<double, double> v0 = d.lev[l].view;                            // -(LU)^-1 F y in level rows
    v0.k = 0;
    launch_couple<double, double>(v0, h->zeros, X, d.partial, d.counter, d.u, st);   // tail = E (LU)^-1 F y
    GEMSLR_CUDA(cudaMemcpyAsync(out, X + hl.e, 8 * s, cudaMemcpyDeviceToDevice, st));
}

void read_ctl(gemslr_ctx *h, cudaStream_t st) {
    GEMSLR_CUDA(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
}

void write_ctl(gemslr_ctx *h, cudaStream_t st) {
    GEMSLR_CUDA(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(KrylovCtl), cudaMemcpyHostToDevice, st));
}

double read_scalar(gemslr_ctx *h, const double *dev, cudaStream_t st) {
    GEMSLR_CUDA(cudaMemcpyAsync(h->n2_host, dev, 8, cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
    return h->n2_host[0];
}

// 2u - 1 from splitmix64(seed): the seeded Arnoldi start vector.
std::vector<double> start_vector(uint64_t seed, int64_t s) {
    std::vector<double> v = splitmix_uniform01(seed, s);
    for (double &x : v) x = 2.0 * x - 1.0;
    return v;
}

// Low-rank correction of level l by thick-restart (Krylov-Schur) Arnoldi on
// G_hat_l with classical Gram-Schmidt and one forced re-orthogonalisation.
// Cycle m = 2k; the wanted subspace is kept on restart; converged when
// ||beta * Q[m-1, :k]||_2 <= tol * min |theta_i| (every Ritz value to ~two
// digits, Sec. 5 set-up); s_l <= m: dense G_hat and its full Schur form.

// Randomized block set-up of level l's correction (Sec. 6 future work): an
// s x b block (b = 2k) of 2u - 1 from splitmix64(1000 + l), column after
// column; Y = G_hat Omega and lowrank_power passes of Q = orth(Y),
// Y = G_hat Q; Q = orth(Y) by classical Gram-Schmidt with a second pass (the
// Arnoldi's kernels, column by column); Z = G_hat Q and B = Q^T Z; the wanted
// part of B's Schur form gives W = Q U_k and H (same selection as the
// Arnoldi).  A column that Gram-Schmidt annihilates ends the block early.
void build_lowrank_randomized(gemslr_ctx *h, int l, int k, int b, cudaStream_t st) {
    HostLevel &hl = h->host.lev[l];
    const int64_t s = h->host.n - hl.e;
    double *V = (double *)h->arena.alloc(8 * (size_t)s * (b + 1));
    double *Y = (double *)h->arena.alloc(8 * (size_t)s * b);
    double *w = (double *)h->arena.alloc(8 * (size_t)s);
    double *Hd = (double *)h->arena.alloc(8 * (size_t)(b + 1) * b);
    double *Bd = (double *)h->arena.alloc(8 * (size_t)b * b);
    double *Qd = (double *)h->arena.alloc(8 * (size_t)b * (k + 2));
    double *W2 = (double *)h->arena.alloc(8 * (size_t)s * (k + 2));
    {
        std::vector<double> u = splitmix_uniform01(1000 + (uint64_t)l, s * b);
        for (double &x : u) x = 2.0 * x - 1.0;
        GEMSLR_CUDA(cudaMemcpyAsync(V, u.data(), 8 * (size_t)s * b, cudaMemcpyHostToDevice, st));
    }
    int bb = b;                                      // columns of the current orthonormal block
    auto apply_block = [&](const double *X, int cols) {
        for (int c = 0; c < cols; ++c) g_hat(h, l, X + (size_t)c * s, Y + (size_t)c * s, st);
    };
    // Q = orth(Y[:, :cols]) into V; returns the number of columns kept
    auto orth = [&](int cols) {
        launch_norm2(s, Y, h->partial, h->counter, h->n2, h->red_grid, st);
        launch_scale_by_norm(s, Y, h->n2, V, st);
        KrylovCtl c{};
        c.j = 0;
        c.m = cols;
        c.givens = 0;
        c.force_reorth = 1;
        c.maxit = 1 << 30;
        *h->ctl_host = c;
        write_ctl(h, st);
        GEMSLR_CUDA(cudaMemsetAsync(Hd, 0, 8 * (size_t)(b + 1) * b, st));
        for (int j = 1; j < cols; ++j) {
            GEMSLR_CUDA(cudaMemcpyAsync(w, Y + (size_t)j * s, 8 * s, cudaMemcpyDeviceToDevice, st));
            launch_gs_dots(s, V, s, w, h->partial, h->counter, h->ctl, Hd, nullptr, nullptr, nullptr, h->h2,
                           h->red_grid, st);
            launch_gs_sub(s, V, s, w, h->partial, h->counter, h->ctl, Hd, nullptr, nullptr, nullptr, h->h2,
                          h->red_grid, st);
            launch_gs_sub2(s, V, s, w, h->h2, h->partial, h->counter, h->ctl, Hd, nullptr, nullptr, nullptr,
                           h->red_grid, st);
            launch_gs_scale(s, V, s, w, h->ctl, nullptr, st);
            launch_gs_next(h->ctl, st);
            read_ctl(h, st);
            if (h->ctl_host->breakdown) return j;    // column j lies in the span of the ones before
        }
        return cols;
    };
    apply_block(V, bb);
    for (int it = 0; it < h->opt.lowrank_power; ++it) {
        bb = orth(bb);
        apply_block(V, bb);
    }
    bb = orth(bb);
    apply_block(V, bb);                              // Z = G_hat Q (in Y)
    launch_gram(s, bb, V, Y, Bd, st);
    std::vector<double> B((size_t)bb * bb), Q, Tk, tre, tim;
    GEMSLR_CUDA(cudaMemcpyAsync(B.data(), Bd, 8 * B.size(), cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
    const int keff = schur_wanted(B, bb, std::min(k, bb), Q, Tk, tre, tim);
    GEMSLR_CUDA(cudaMemcpyAsync(Qd, Q.data(), 8 * (size_t)bb * keff, cudaMemcpyHostToDevice, st));
    launch_basis_rotate(s, V, s, bb, Qd, keff, W2, st);
    hl.k = keff;
    hl.W.resize((size_t)s * keff);
    GEMSLR_CUDA(cudaMemcpyAsync(hl.W.data(), W2, 8 * (size_t)s * keff, cudaMemcpyDeviceToHost, st));
    GEMSLR_CUDA(cudaStreamSynchronize(st));
    hl.H = correction_matrix(Tk, keff);
}

void build_lowrank(gemslr_ctx *h, int l, cudaStream_t st) {
    HostLevel &hl = h->host.lev[l];
    const int64_t s = h->host.n - hl.e;
    int k = std::max(0, hl.rank_req);
    hl.k = 0;
    hl.W.clear();
    hl.H.clear();
    if (k == 0 || s == 0) return;
    const int m = 2 * k;
    std::vector<double> Q, Tk, tre, tim;
    if (s <= m) {
        std::vector<double> G((size_t)s * s), e(s, 0.0);
        double *ed = (double *)h->arena.alloc(8 * s), *gd = (double *)h->arena.alloc(8 * s);
        for (int64_t i = 0; i < s; ++i) {
            e.assign(s, 0.0);
            e[i] = 1.0;
            GEMSLR_CUDA(cudaMemcpyAsync(ed, e.data(), 8 * s, cudaMemcpyHostToDevice, st));
            g_hat(h, l, ed, gd, st);
            GEMSLR_CUDA(cudaMemcpyAsync(G.data() + (size_t)i * s, gd, 8 * s, cudaMemcpyDeviceToHost, st));
            GEMSLR_CUDA(cudaStreamSynchronize(st));
        }
        const int keff = schur_wanted(G, (int)s, k, Q, Tk, tre, tim);
        hl.k = keff;
        hl.W.assign(Q.begin(), Q.begin() + (size_t)s * keff);
        hl.H = correction_matrix(Tk, keff);
        return;
    }
    if (m + 1 > kMaxCols) fail(GEMSLR_ERR_ARG, "rank too large for the Arnoldi workspace");
    if (h->opt.lowrank_method == GEMSLR_LOWRANK_RANDOMIZED) {
        build_lowrank_randomized(h, l, k, m, st);
        return;
    }
    double *V = (double *)h->arena.alloc(8 * (size_t)s * (m + 1));
    double *W2 = (double *)h->arena.alloc(8 * (size_t)s * (k + 2));
    double *w = (double *)h->arena.alloc(8 * (size_t)s);
    double *Hd = (double *)h->arena.alloc(8 * (size_t)(m + 1) * m);
    double *Qd = (double *)h->arena.alloc(8 * (size_t)m * (k + 2));
    std::vector<double> v1 = start_vector(1000 + (uint64_t)l, s);
    double nv = 0.0;
    for (double x : v1) nv += x * x;
    nv = std::sqrt(nv);
    for (double &x : v1) x /= nv;
    GEMSLR_CUDA(cudaMemcpyAsync(V, v1.data(), 8 * s, cudaMemcpyHostToDevice, st));
    std::vector<double> Hb((size_t)(m + 1) * m, 0.0);
    GEMSLR_CUDA(cudaMemsetAsync(Hd, 0, 8 * (size_t)(m + 1) * m, st));
    const double tol = h->opt.arnoldi_tol > 0 ? h->opt.arnoldi_tol : 1e-2;
    const int maxc = h->opt.arnoldi_max_cycles > 0 ? h->opt.arnoldi_max_cycles : 20;
    int p = 0;
    for (int cycle = 0; cycle < maxc; ++cycle) {
        KrylovCtl c{};
        c.j = p;
        c.m = m;
        c.givens = 0;
        c.force_reorth = 1;
        c.maxit = 1 << 30;
        *h->ctl_host = c;
        write_ctl(h, st);
        int mm = m;
        bool broke = false;
        double beta = 0.0;
        for (int j = p; j < m; ++j) {
            g_hat(h, l, V + (size_t)j * s, w, st);
            launch_gs_dots(s, V, s, w, h->partial, h->counter, h->ctl, Hd, nullptr, nullptr, nullptr, h->h2, h->red_grid,
                           st);
            launch_gs_sub(s, V, s, w, h->partial, h->counter, h->ctl, Hd, nullptr, nullptr, nullptr, h->h2,
                          h->red_grid, st);
            launch_gs_sub2(s, V, s, w, h->h2, h->partial, h->counter, h->ctl, Hd, nullptr, nullptr, nullptr,
                           h->red_grid, st);
            launch_gs_scale(s, V, s, w, h->ctl, nullptr, st);
            launch_gs_next(h->ctl, st);
            read_ctl(h, st);
            beta = h->ctl_host->beta;
            if (h->ctl_host->breakdown) { mm = j + 1; broke = true; beta = 0.0; break; }
        }
        GEMSLR_CUDA(cudaMemcpyAsync(Hb.data(), Hd, 8 * Hb.size(), cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaStreamSynchronize(st));
        std::vector<double> Hm((size_t)mm * mm);
        for (int j = 0; j < mm; ++j)
            for (int i = 0; i < mm; ++i) Hm[i + (size_t)j * mm] = Hb[i + (size_t)j * (m + 1)];
        const int keff = schur_wanted(Hm, mm, k, Q, Tk, tre, tim);
        double res = 0.0, tmin = INFINITY;
        for (int t = 0; t < keff; ++t) {
            const double q = beta * Q[(mm - 1) + (size_t)t * mm];
            res += q * q;
            tmin = std::min(tmin, std::hypot(tre[t], tim[t]));
        }
        res = std::sqrt(res);
        const bool ok = broke || res <= tol * tmin;
        GEMSLR_CUDA(cudaMemcpyAsync(Qd, Q.data(), 8 * (size_t)mm * keff, cudaMemcpyHostToDevice, st));
        launch_basis_rotate(s, V, s, mm, Qd, keff, W2, st);
        if (ok || cycle == maxc - 1) {
            hl.k = keff;
            hl.W.resize((size_t)s * keff);
            GEMSLR_CUDA(cudaMemcpyAsync(hl.W.data(), W2, 8 * (size_t)s * keff, cudaMemcpyDeviceToHost, st));
            GEMSLR_CUDA(cudaStreamSynchronize(st));
            hl.H = correction_matrix(Tk, keff);
            return;
        }
        // thick restart: V[:, :keff] = V Q, V[:, keff] = v_{m+1}
        GEMSLR_CUDA(cudaMemcpyAsync(V + (size_t)keff * s, V + (size_t)mm * s, 8 * s, cudaMemcpyDeviceToDevice, st));
        GEMSLR_CUDA(cudaMemcpyAsync(V, W2, 8 * (size_t)s * keff, cudaMemcpyDeviceToDevice, st));
        std::fill(Hb.begin(), Hb.end(), 0.0);
        for (int b = 0; b < keff; ++b) {
            for (int a = 0; a < keff; ++a) Hb[a + (size_t)b * (m + 1)] = Tk[a + (size_t)b * keff];
            Hb[keff + (size_t)b * (m + 1)] = beta * Q[(mm - 1) + (size_t)b * mm];
        }
        GEMSLR_CUDA(cudaMemcpyAsync(Hd, Hb.data(), 8 * Hb.size(), cudaMemcpyHostToDevice, st));
        p = keff;
    }
}

void finish_setup(gemslr_ctx *h, bool compute_lowrank) {
    // this host thread's own stream: set-ups of several systems on several
    // threads (the batched set-up) overlap their per-step host round trips
    cudaStream_t st = cudaStreamPerThread;
    const int64_t n = h->host.n;
    const Csr &A = h->host.Ahat;
    h->A_rp = h->arena.upload(A.rp);
    h->A_ci = h->arena.upload(A.ci);
    h->A_v = h->arena.upload(A.v);
    const double avg = n ? (double)A.nnz() / n : 0.0;
    h->spmv_lanes = avg <= 3 ? 2 : (avg <= 8 ? 4 : (avg <= 24 ? 8 : 16));
    h->perm = h->arena.upload(h->host.perm);
    h->zeros = (double *)h->arena.alloc(8 * std::max<int64_t>(n, 1));
    GEMSLR_CUDA(cudaMemset(h->zeros, 0, 8 * std::max<int64_t>(n, 1)));
    const int limit = smem_optin();
    if (h->host.cplx) {            // complex shift (Sec. 5.2.3): complex hierarchy only
        ensure_krylov(h, 8);
        h->z = z_create(h->host, h->arena, h->opt, h->A_rp, h->A_ci, h->A_v, h->perm, limit, sm_count(),
                        compute_lowrank);
        return;
    }
    upload_hierarchy<double, double>(h->host, h->arena, h->d64, limit);
    ensure_krylov(h, 8);
    if (compute_lowrank) {
        for (int l = (int)h->host.lev.size() - 1; l >= 0; --l) {   // bottom-up (Sec. 4.2)
            build_lowrank(h, l, st);
            set_lowrank<double, double>(h->d64.lev[l], h->host.lev[l], h->arena);
        }
    }
    if (h->opt.precision == GEMSLR_PREC_MIXED) {
        upload_hierarchy<float, __nv_bfloat16>(h->host, h->arena, h->d32, limit);
        h->mixed = true;
    }
    GEMSLR_CUDA(cudaDeviceSynchronize());
}

// ---- FGMRES (Sec. 4.1) ---------------------------------------------------------------
// One Arnoldi step on fixed buffers: z = M^{-1} vin, w = A z with z stored as
// Z[:, j], Gram-Schmidt against V[:, :j+1], Givens update, and the next basis
// vector written to V[:, j+1] and to vin.
void fgmres_step(gemslr_ctx *h, cudaStream_t st) {
    const int64_t n = h->host.n;
    apply_perm(h, h->vin, h->zout, st);
    if (h->spmv_lanes <= 8) {       // short rows: the product is fused into the first pass
        ProfScope ps("spmv_gs_dots", st);
        launch_gs_spmv_dots(n, h->A_rp, h->A_ci, h->A_v, h->zout, h->Z, h->V, n, h->w, h->partial, h->counter,
                            h->ctl, h->Hs, h->cs, h->sn, h->g, h->h2, h->red_grid, st);
    } else {
        {
            ProfScope ps("spmv_A", st);
            launch_spmv(n, h->A_rp, h->A_ci, h->A_v, h->zout, nullptr, h->w, h->spmv_lanes, st, h->Z, h->ctl);
        }
        ProfScope ps("gs_dots", st);
        launch_gs_dots(n, h->V, n, h->w, h->partial, h->counter, h->ctl, h->Hs, h->cs, h->sn, h->g, h->h2,
                       h->red_grid, st);
    }
    {
        ProfScope ps("gs_sub", st);
        launch_gs_sub(n, h->V, n, h->w, h->partial, h->counter, h->ctl, h->Hs, h->cs, h->sn, h->g, h->h2,
                      h->red_grid, st, h->vin);
    }
    {
        ProfScope ps("gs_sub2", st);
        launch_gs_sub2(n, h->V, n, h->w, h->h2, h->partial, h->counter, h->ctl, h->Hs, h->cs, h->sn, h->g,
                       h->red_grid, st);
        launch_gs_scale(n, h->V, n, h->w, h->ctl, h->vin, st);
    }
}

// FGMRES with delayed reorthogonalisation applies only where M^{-1} is linear
// (not with the learned stage) and the fused product suits A (short rows).
bool use_dcgs(const gemslr_ctx *h) {
    const bool learned = (h->d64.learned && h->d64.learned->enabled) || (h->d32.learned && h->d32.learned->enabled);
    const bool inner = h->d64.inner.k > 0 || h->d32.inner.k > 0;     // Alg. 2 step 9 makes M^{-1} nonlinear
    return !learned && !inner && h->spmv_lanes <= 8;
}

DgsBufs dgs_bufs(gemslr_ctx *h) {
    DgsBufs B;
    B.Hraw = h->Hraw;
    B.Hrot = h->Hs;
    B.cs = h->cs;
    B.sn = h->sn;
    B.g = h->g;
    B.R = h->Rz;
    B.a = h->da;
    B.coef = h->dcoef;
    B.apre = h->dapre;
    B.hprev = h->dhprev;
    return B;
}

// One step with delayed reorthogonalisation: z = M^{-1} vt, the fused product
// and reduction, then the basis column and the next direction.
void fgmres_step_d(gemslr_ctx *h, cudaStream_t st) {
    const int64_t n = h->host.n;
    const DgsBufs B = dgs_bufs(h);
    if (!h->aux_stream) {
        GEMSLR_CUDA(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
        GEMSLR_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        GEMSLR_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        GEMSLR_CUDA(cudaEventCreateWithFlags(&h->ev_fork2, cudaEventDisableTiming));
        GEMSLR_CUDA(cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming));
    }
    // the previous step's reorthogonalisation runs beside z = M^{-1} vt_j on
    // the SMs the level-0 substitutions leave free (one CTA per SM, none
    // sharing an SM with a substitution CTA); the reduction below needs both
    const int nb0 = h->host.lev.empty() ? 0 : (int)h->host.lev[0].bp.size() - 1;
    const int fix_grid = std::max(16, h->red_grid - nb0);
    GEMSLR_CUDA(cudaEventRecord(h->ev_fork, st));
    GEMSLR_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
    {
        ProfScope ps("dgs_fix_adots", h->aux_stream);
        launch_dgs_fix_adots(n, h->V, n, h->vin, h->partial2, h->counter2, h->ctl, B, fix_grid, h->aux_stream);
    }
    GEMSLR_CUDA(cudaEventRecord(h->ev_join, h->aux_stream));
    apply_perm(h, h->vin, h->zout, st);
    GEMSLR_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
    {
        ProfScope ps("dgs_spmv_dots", st);
        launch_dgs_dots(n, h->A_rp, h->A_ci, h->A_v, h->zout, h->Z, h->V, n, h->vin, h->w, h->partial, h->counter,
                        h->ctl, B, h->red_grid, st);
    }
    // the Hessenberg bookkeeping and the stopping test beside the next direction
    GEMSLR_CUDA(cudaEventRecord(h->ev_fork2, st));
    GEMSLR_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_fork2, 0));
    {
        ProfScope ps("dgs_tail", h->aux_stream);
        launch_dgs_tail(h->ctl, B, h->aux_stream);
    }
    GEMSLR_CUDA(cudaEventRecord(h->ev_join2, h->aux_stream));
    {
        ProfScope ps("dgs_next", st);
        launch_dgs_next(n, h->V, n, h->vin, h->w, h->ctl, B, st);
    }
    GEMSLR_CUDA(cudaStreamWaitEvent(st, h->ev_join2, 0));
}

// End of a delayed cycle: close the last column, y = Hrot^{-1} g, y = R^{-1} y,
// x += Zt y, r = b - A x, ||r||^2 into n2[1].
void fgmres_cycle_end_d(gemslr_ctx *h, cudaStream_t st) {
    const int64_t n = h->host.n;
    const DgsBufs B = dgs_bufs(h);
    launch_dgs_fix(n, h->V, n, h->ctl, B, 0, 8 * h->red_grid, false, st);   // the last step's v_j
    launch_dgs_close(n, h->V, n, h->vin, h->partial, h->counter, h->ctl, B, h->red_grid, st);
    launch_lsq2(h->ctl, h->Hs, h->g, h->Rz, h->y, st);
    launch_update_x(n, h->Z, n, h->ctl, h->y, h->xh, st);
    launch_spmv(n, h->A_rp, h->A_ci, h->A_v, h->xh, h->bh, h->r, h->spmv_lanes, st);
    launch_norm2(n, h->r, h->partial, h->counter, h->n2 + 1, h->red_grid, st);
}

// End of a cycle: x += Z y, r = b - A x, ||r||^2 into n2[1].
void fgmres_cycle_end(gemslr_ctx *h, cudaStream_t st) {
    const int64_t n = h->host.n;
    launch_lsq(h->ctl, h->Hs, h->g, h->y, st);
    launch_update_x(n, h->Z, n, h->ctl, h->y, h->xh, st);
    launch_spmv(n, h->A_rp, h->A_ci, h->A_v, h->xh, h->bh, h->r, h->spmv_lanes, st);
    launch_norm2(n, h->r, h->partial, h->counter, h->n2 + 1, h->red_grid, st);
}

// Host-driven loop (used while profiling): the host reads the control block
// after every step and every cycle.
void fgmres_host_loop(gemslr_ctx *h, int m, bool dcgs, cudaStream_t st) {
    const int64_t n = h->host.n;
    launch_zero(n, h->xh, st);
    GEMSLR_CUDA(cudaMemcpyAsync(h->r, h->bh, 8 * n, cudaMemcpyDeviceToDevice, st));
    GEMSLR_CUDA(cudaMemcpyAsync(h->n2 + 1, h->n2, 8, cudaMemcpyDeviceToDevice, st));
    while (true) {
        launch_cycle_start(h->ctl, h->g, h->n2 + 1, st);
        launch_scale_by_norm(n, h->r, h->n2 + 1, h->V, st, h->vin);
        for (int j = 0; j < m; ++j) {
            if (dcgs) fgmres_step_d(h, st);
            else fgmres_step(h, st);
            launch_gs_next(h->ctl, st);
            read_ctl(h, st);
            if (h->ctl_host->stop) break;
        }
        if (dcgs) fgmres_cycle_end_d(h, st);
        else fgmres_cycle_end(h, st);
        const double rn = std::sqrt(read_scalar(h, h->n2 + 1, st));
        read_ctl(h, st);
        KrylovCtl &k = *h->ctl_host;
        k.rnorm = rn;
        bool again = true;
        if (!std::isfinite(rn) || k.nonfinite) { k.nonfinite = 1; again = false; }
        else if (rn <= k.tol_abs) { k.converged = 1; again = false; }
        else if (k.iters >= k.maxit) again = false;
        else k.restarts += 1;
        write_ctl(h, st);
        if (!again) break;
    }
    read_ctl(h, st);
}

}  // namespace

namespace gemslr {
// Add a WHILE conditional node at the current capture position of `cs`;
// returns its body graph.
cudaGraph_t capture_while_node(cudaStream_t cs, cudaGraphConditionalHandle handle) {
    cudaStreamCaptureStatus status;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    GEMSLR_CUDA(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = handle;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    GEMSLR_CUDA(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p));
    GEMSLR_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return p.conditional.phGraph_out[0];
}
}  // namespace gemslr

namespace {

// The whole solve as one CUDA graph: prologue, then
//   WHILE (cycle) { cycle start; WHILE (step) { FGMRES step }; cycle end }
// with both conditions set by device kernels from the control block, so a
// solve needs no host round trip.  Built once per restart length.
bool ensure_solve_graph(gemslr_ctx *h, int m, bool dcgs) {
    if (h->graph_failed) return false;
    if (h->graph_exec && h->graph_m == m && h->graph_dcgs == dcgs) return true;
    try {
        if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
        if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
        if (!h->cap_stream) GEMSLR_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaStream_t cs = h->cap_stream;
        const int64_t n = h->host.n;
        const uint64_t k0 = launches_total();
        cudaGraph_t g;
        GEMSLR_CUDA(cudaGraphCreate(&g, 0));
        h->graph = g;
        cudaGraphConditionalHandle hc;
        GEMSLR_CUDA(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
        GEMSLR_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        launch_zero(n, h->xh, cs);
        GEMSLR_CUDA(cudaMemcpyAsync(h->r, h->bh, 8 * n, cudaMemcpyDeviceToDevice, cs));
        GEMSLR_CUDA(cudaMemcpyAsync(h->n2 + 1, h->n2, 8, cudaMemcpyDeviceToDevice, cs));
        cudaGraph_t body_cycle = capture_while_node(cs, hc);
        GEMSLR_CUDA(cudaStreamEndCapture(cs, &g));
        const uint64_t k1 = launches_total();
        cudaGraphConditionalHandle hs;
        GEMSLR_CUDA(cudaGraphConditionalHandleCreate(&hs, body_cycle, 1, cudaGraphCondAssignDefault));
        GEMSLR_CUDA(cudaStreamBeginCaptureToGraph(cs, body_cycle, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        launch_cycle_start_g(h->ctl, h->g, h->n2 + 1, hs, cs);
        launch_scale_by_norm(n, h->r, h->n2 + 1, h->V, cs, h->vin);
        cudaGraph_t body_step = capture_while_node(cs, hs);
        if (dcgs) fgmres_cycle_end_d(h, cs);
        else fgmres_cycle_end(h, cs);
        launch_cycle_end_g(h->ctl, h->n2 + 1, hc, cs);
        GEMSLR_CUDA(cudaStreamEndCapture(cs, &body_cycle));
        const uint64_t k2 = launches_total();
        GEMSLR_CUDA(cudaStreamBeginCaptureToGraph(cs, body_step, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        if (dcgs) fgmres_step_d(h, cs);
        else fgmres_step(h, cs);
        launch_step_end_g(h->ctl, hs, cs);
        GEMSLR_CUDA(cudaStreamEndCapture(cs, &body_step));
        const uint64_t k3 = launches_total();
        GEMSLR_CUDA(cudaGraphInstantiate(&h->graph_exec, g, 0));
        h->graph_k_top = k1 - k0;
        h->graph_k_cycle = k2 - k1;
        h->graph_k_step = k3 - k2;
        count_launch(-(int)(k3 - k0));      // capture launches nothing
        h->graph_m = m;
        h->graph_dcgs = dcgs;
        return true;
    } catch (const Error &e) {
        cudaGetLastError();
        h->graph_failed = true;
        if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
        if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
        return false;
    }
}

gemslr_status guard(const std::function<void()> &fn) {
    try {
        fn();
        return GEMSLR_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return GEMSLR_ERR_NOMEM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return GEMSLR_ERR_ARG;
    }
}

gemslr_options normalized(const gemslr_options *opt) {
    gemslr_options o;
    gemslr_default_options(&o);
    if (opt) o = *opt;
    if (o.ilu_kind != GEMSLR_ILU0 && o.ilu_kind != GEMSLR_ILUT && o.ilu_kind != GEMSLR_ILU0_DEVICE &&
        o.ilu_kind != GEMSLR_ILUT_DEVICE)
        fail(GEMSLR_ERR_ARG, "unknown ilu_kind");
    if (o.ilu_kind == GEMSLR_ILUT_DEVICE && (o.ilut_lfil < 0 || o.ilut_lfil > 64))
        fail(GEMSLR_ERR_ARG, "device ILUT needs 0 <= ilut_lfil <= 64");
    if (o.precision != GEMSLR_PREC_FP64 && o.precision != GEMSLR_PREC_MIXED) fail(GEMSLR_ERR_ARG, "unknown precision");
    if (o.ilut_tau < 0) fail(GEMSLR_ERR_ARG, "ilut_tau must be >= 0");
    for (int l = 0; l < GEMSLR_MAX_LEVELS; ++l)
        if (o.rank[l] < 0 || 2 * o.rank[l] + 1 > kMaxCols || o.rank[l] + 2 > kMaxRank)
            fail(GEMSLR_ERR_ARG, "rank out of range (0..79)");
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr))
        fail(GEMSLR_ERR_ARG, "dev_alloc and dev_free must be given together");
    if (o.lowrank_method != GEMSLR_LOWRANK_ARNOLDI && o.lowrank_method != GEMSLR_LOWRANK_RANDOMIZED)
        fail(GEMSLR_ERR_ARG, "unknown lowrank_method");
    if (o.lowrank_power < 0 || o.lowrank_power > 16) fail(GEMSLR_ERR_ARG, "lowrank_power must be in 0..16");
    if (!std::isfinite(o.shift)) fail(GEMSLR_ERR_ARG, "shift must be finite");
    if (o.shift != 0.0 && (o.precision != GEMSLR_PREC_FP64 || o.lowrank_method != GEMSLR_LOWRANK_ARNOLDI ||
                           o.ilu_kind == GEMSLR_ILU0_DEVICE || o.ilu_kind == GEMSLR_ILUT_DEVICE))
        fail(GEMSLR_ERR_UNSUPPORTED, "the complex shift needs FP64, a host ILU and the Arnoldi set-up");
    return o;
}

}  // namespace

namespace gemslr {
// Single-system setup (factors and low-rank terms, FP64) kept on the host; the
// device copy used for the Arnoldi products is released afterwards.
void setup_single_host(const gemslr_csr *A, const gemslr_partition *part, const gemslr_options *opt, Hierarchy &out) {
    std::unique_ptr<gemslr_ctx> h(new gemslr_ctx());
    h->opt = normalized(opt);
    h->arena.set_allocator(h->opt.dev_alloc, h->opt.dev_free, h->opt.alloc_ctx);
    h->opt.precision = GEMSLR_PREC_FP64;
    Csr M = csr_from_abi(A);
    build_levels(M, part, &h->opt, h->host);
    finish_setup(h.get(), true);
    out = std::move(h->host);
}

// Host hierarchy whose levels are sliced from the partition (A permuted, E and
// F formed) but whose factors all come from f: nothing is factored.
void hierarchy_from_factors(const gemslr_csr *A, const gemslr_partition *part, const gemslr_factors *f,
                            const gemslr_options &opt, Hierarchy &H) {
    if (!f) fail(GEMSLR_ERR_ARG, "NULL factors");
    Csr M = csr_from_abi(A);
    gemslr_options o = opt;
    o.ilu_kind = GEMSLR_ILU0;       // cheap placeholder factorisation, replaced below
    o.shift = 0.0;
    for (int l = 0; l < GEMSLR_MAX_LEVELS; ++l) o.rank[l] = 0;
    build_levels(M, part, &o, H);
    // imaginary parts (complex factors): copied into vi / Wi / Hi, NULL: none
    auto imag = [&H](Csr &T, const double *im) {
        if (!im) return;
        T.vi.assign(im, im + T.nnz());
        H.cplx = true;
    };
    if (f->nlev != H.nlev || (H.nlev > 1 && !f->levels)) fail(GEMSLR_ERR_ARG, "factor level count mismatch");
    for (int l = 0; l < H.nlev - 1; ++l) {
        const gemslr_level_factors &lf = f->levels[l];
        HostLevel &hl = H.lev[l];
        const int64_t d = hl.e - hl.s, s = H.n - hl.e;
        hl.L = csr_from_mat(lf.L);
        hl.U = csr_from_mat(lf.U);
        hl.E = csr_from_mat(lf.E);
        hl.F = csr_from_mat(lf.F);
        if (hl.L.nrows != d || hl.U.nrows != d || hl.E.nrows != s || hl.E.ncols != d || hl.F.nrows != d ||
            hl.F.ncols != s)
            fail(GEMSLR_ERR_ARG, "factor shapes do not match the partition at level " + std::to_string(l));
        if (lf.k < 0 || lf.k + 2 > kMaxRank) fail(GEMSLR_ERR_ARG, "rank out of range");
        hl.k = lf.k;
        hl.W.clear();
        hl.H.clear();
        if (lf.k > 0) {
            if (!lf.W || !lf.H) fail(GEMSLR_ERR_ARG, "W/H missing");
            hl.W.assign(lf.W, lf.W + (size_t)s * lf.k);
            hl.H.assign(lf.H, lf.H + (size_t)lf.k * lf.k);
            hl.Wi.clear();
            hl.Hi.clear();
            if (lf.W_im) { hl.Wi.assign(lf.W_im, lf.W_im + (size_t)s * lf.k); H.cplx = true; }
            if (lf.H_im) { hl.Hi.assign(lf.H_im, lf.H_im + (size_t)lf.k * lf.k); H.cplx = true; }
        }
        imag(hl.L, lf.L_im);
        imag(hl.U, lf.U_im);
    }
    H.last.L = csr_from_mat(f->last_L);
    H.last.U = csr_from_mat(f->last_U);
    imag(H.last.L, f->last_L_im);
    imag(H.last.U, f->last_U_im);
    if (H.last.L.nrows != H.n - H.last.s || H.last.U.nrows != H.n - H.last.s)
        fail(GEMSLR_ERR_ARG, "last-level factor shape mismatch");
}
}  // namespace gemslr

extern "C" {

void gemslr_default_options(gemslr_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->ilu_kind = GEMSLR_ILUT;
    opt->ilut_tau = 1e-3;
    opt->ilut_lfil = 10;
    opt->precision = GEMSLR_PREC_FP64;
    opt->arnoldi_tol = 1e-2;
    opt->arnoldi_max_cycles = 20;
    opt->lowrank_method = GEMSLR_LOWRANK_ARNOLDI;
    opt->lowrank_power = 1;
    opt->shift = 0.0;
}

const char *gemslr_last_error(void) { return g_last_error.c_str(); }

gemslr_status gemslr_partition_geometric(const gemslr_csr *A, const int32_t *coords, int32_t nlev, int32_t p,
                                         int32_t p_last, int32_t *perm, int64_t *level_ptr, int32_t *nblk,
                                         int64_t *block_ptr) {
    return guard([&] {
        if (!perm || !level_ptr || !nblk || !block_ptr) fail(GEMSLR_ERR_ARG, "NULL output array");
        Csr M = csr_from_abi(A);
        std::vector<int32_t> pv, nb;
        std::vector<int64_t> lp, bp;
        partition_geometric(M, coords, nlev, p, p_last, pv, lp, nb, bp);
        std::copy(pv.begin(), pv.end(), perm);
        std::copy(lp.begin(), lp.end(), level_ptr);
        std::copy(nb.begin(), nb.end(), nblk);
        std::copy(bp.begin(), bp.end(), block_ptr);
    });
}

gemslr_status gemslr_local_order(int64_t n, const int32_t *coords, const gemslr_partition *part, int32_t first_level,
                                 int32_t *perm_out) {
    return guard([&] {
        if (n < 0 || !coords || !part || !perm_out || !part->perm || !part->level_ptr || !part->nblk ||
            !part->block_ptr || part->nlev < 1)
            fail(GEMSLR_ERR_ARG, "NULL argument or empty partition");
        std::vector<int32_t> pv(part->perm, part->perm + n), nb(part->nblk, part->nblk + part->nlev);
        std::vector<int64_t> lp(part->level_ptr, part->level_ptr + part->nlev + 1);
        int64_t nbp = 0;
        for (int32_t v : nb) {
            if (v < 1) fail(GEMSLR_ERR_PARTITION, "every level needs at least one block");
            nbp += v + 1;
        }
        std::vector<int64_t> bp(part->block_ptr, part->block_ptr + nbp);
        if (lp[0] != 0 || lp.back() != n) fail(GEMSLR_ERR_PARTITION, "level_ptr must run from 0 to n");
        local_order(coords, n, lp, nb, bp, first_level, pv);
        std::copy(pv.begin(), pv.end(), perm_out);
    });
}

gemslr_status gemslr_setup(const gemslr_csr *A, const gemslr_partition *part, const gemslr_options *opt,
                           gemslr_handle *out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out) fail(GEMSLR_ERR_ARG, "out is NULL");
        auto t0 = std::chrono::steady_clock::now();
        std::unique_ptr<gemslr_ctx> h(new gemslr_ctx());
        GEMSLR_CUDA(cudaGetDevice(&h->dev));
        h->opt = normalized(opt);
        h->arena.set_allocator(h->opt.dev_alloc, h->opt.dev_free, h->opt.alloc_ctx);
        Csr M = csr_from_abi(A);
        build_levels(M, part, &h->opt, h->host);
        finish_setup(h.get(), true);
        h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = h.release();
    });
}

gemslr_status gemslr_setup_from_factors(const gemslr_csr *A, const gemslr_partition *part, const gemslr_factors *f,
                                        const gemslr_options *opt, gemslr_handle *out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !f) fail(GEMSLR_ERR_ARG, "NULL argument");
        auto t0 = std::chrono::steady_clock::now();
        std::unique_ptr<gemslr_ctx> h(new gemslr_ctx());
        GEMSLR_CUDA(cudaGetDevice(&h->dev));
        h->opt = normalized(opt);
        h->arena.set_allocator(h->opt.dev_alloc, h->opt.dev_free, h->opt.alloc_ctx);
        hierarchy_from_factors(A, part, f, h->opt, h->host);
        Hierarchy &H = h->host;
        if (H.cplx && h->opt.precision != GEMSLR_PREC_FP64)
            fail(GEMSLR_ERR_UNSUPPORTED, "complex factors need precision FP64");
        finish_setup(h.get(), false);
        if (H.cplx) {
            h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            *out = h.release();
            return;
        }
        for (size_t l = 0; l < H.lev.size(); ++l) set_lowrank<double, double>(h->d64.lev[l], H.lev[l], h->arena);
        if (h->mixed) {
            // rebuild the mixed hierarchy now that W/H are attached
            h->d32 = DevHierarchy<float, __nv_bfloat16>();
            upload_hierarchy<float, __nv_bfloat16>(H, h->arena, h->d32, smem_optin());
        }
        GEMSLR_CUDA(cudaDeviceSynchronize());
        h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = h.release();
    });
}

gemslr_status gemslr_factor_sizes(gemslr_handle h, int64_t *counts, int64_t ncounts) {
    return guard([&] {
        if (!h || !counts) fail(GEMSLR_ERR_ARG, "NULL argument");
        const Hierarchy &H = h->host;
        if (ncounts < 4 + 9 * (int64_t)H.lev.size()) fail(GEMSLR_ERR_ARG, "counts too small");
        counts[0] = H.nlev;
        for (size_t l = 0; l < H.lev.size(); ++l) {
            const HostLevel &hl = H.lev[l];
            int64_t *c = counts + 1 + 9 * l;
            c[0] = hl.L.nnz(); c[1] = hl.U.nnz(); c[2] = hl.E.nnz(); c[3] = hl.F.nnz(); c[4] = hl.k;
            c[5] = hl.e - hl.s; c[6] = H.n - hl.e; c[7] = hl.s; c[8] = hl.e;
        }
        int64_t *c = counts + 1 + 9 * H.lev.size();
        c[0] = H.last.L.nnz(); c[1] = H.last.U.nnz(); c[2] = H.n - H.last.s;
    });
}

static void put_mat(const Csr &M, const gemslr_mat &dst) {
    if (!dst.rowptr || (M.nnz() > 0 && (!dst.colind || !dst.val))) fail(GEMSLR_ERR_ARG, "NULL export buffer");
    std::copy(M.rp.begin(), M.rp.end(), const_cast<int64_t *>(dst.rowptr));
    std::copy(M.ci.begin(), M.ci.end(), const_cast<int32_t *>(dst.colind));
    std::copy(M.v.begin(), M.v.end(), const_cast<double *>(dst.val));
}

gemslr_status gemslr_export_factors(gemslr_handle h, gemslr_factors *f) {
    return guard([&] {
        if (!h || !f || !f->levels) fail(GEMSLR_ERR_ARG, "NULL argument");
        const Hierarchy &H = h->host;
        if (f->nlev != H.nlev) fail(GEMSLR_ERR_ARG, "nlev mismatch");
        // imaginary parts of a complex handle (zeros where a factor has none)
        auto put_im = [&H](const std::vector<double> &im, size_t count, const double *dst) {
            if (!H.cplx) return;
            if (!dst && count > 0) fail(GEMSLR_ERR_ARG, "complex handle: NULL imaginary-part buffer");
            double *d = const_cast<double *>(dst);
            for (size_t i = 0; i < count; ++i) d[i] = im.empty() ? 0.0 : im[i];
        };
        for (size_t l = 0; l < H.lev.size(); ++l) {
            const HostLevel &hl = H.lev[l];
            const gemslr_level_factors &lf = f->levels[l];
            put_mat(hl.L, lf.L);
            put_mat(hl.U, lf.U);
            put_mat(hl.E, lf.E);
            put_mat(hl.F, lf.F);
            put_im(hl.L.vi, (size_t)hl.L.nnz(), lf.L_im);
            put_im(hl.U.vi, (size_t)hl.U.nnz(), lf.U_im);
            const_cast<gemslr_level_factors &>(lf).k = hl.k;
            if (hl.k > 0) {
                if (!lf.W || !lf.H) fail(GEMSLR_ERR_ARG, "NULL W/H buffer");
                std::copy(hl.W.begin(), hl.W.end(), const_cast<double *>(lf.W));
                std::copy(hl.H.begin(), hl.H.end(), const_cast<double *>(lf.H));
                put_im(hl.Wi, hl.W.size(), lf.W_im);
                put_im(hl.Hi, hl.H.size(), lf.H_im);
            }
        }
        put_mat(H.last.L, f->last_L);
        put_mat(H.last.U, f->last_U);
        put_im(H.last.L.vi, (size_t)H.last.L.nnz(), f->last_L_im);
        put_im(H.last.U.vi, (size_t)H.last.U.nnz(), f->last_U_im);
    });
}

// ---- factor files (checkpoint / resume) --------------------------------------------
// Layout (little-endian, as on the supported hosts): the 8 bytes "GEMSLRF1",
// int64 n, int64 nlev, then per Schur level L, U, E, F as CSR records
// (int64 nrows, ncols, nnz; int64 rowptr[nrows+1]; int32 colind[nnz];
// double val[nnz]), int64 k, double W[(n - level_ptr[l+1]) * k],
// double H[k * k]; then the last level's L and U records.
}  // extern "C"
namespace {
constexpr char kFactorMagic[8] = {'G', 'E', 'M', 'S', 'L', 'R', 'F', '1'};

struct FileCloser {
    void operator()(FILE *f) const { if (f) fclose(f); }
};
using FilePtr = std::unique_ptr<FILE, FileCloser>;

void write_all(FILE *f, const void *p, size_t bytes) {
    if (bytes && fwrite(p, 1, bytes, f) != bytes) fail(GEMSLR_ERR_ARG, "writing the factor file failed");
}
void read_all(FILE *f, void *p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) fail(GEMSLR_ERR_ARG, "factor file truncated or unreadable");
}
void write_csr(FILE *f, const Csr &m) {
    const int64_t hdr[3] = {m.nrows, m.ncols, m.nnz()};
    write_all(f, hdr, sizeof(hdr));
    write_all(f, m.rp.data(), sizeof(int64_t) * m.rp.size());
    write_all(f, m.ci.data(), sizeof(int32_t) * m.ci.size());
    write_all(f, m.v.data(), sizeof(double) * m.v.size());
}
// Reads one CSR record into m; `limit` bounds every size read from the file.
void read_csr(FILE *f, Csr &m, int64_t limit) {
    int64_t hdr[3];
    read_all(f, hdr, sizeof(hdr));
    if (hdr[0] < 0 || hdr[1] < 0 || hdr[2] < 0 || hdr[0] > limit || hdr[1] > limit || hdr[2] > limit * limit)
        fail(GEMSLR_ERR_ARG, "corrupt factor file (matrix sizes)");
    m.nrows = hdr[0];
    m.ncols = hdr[1];
    m.rp.resize(hdr[0] + 1);
    m.ci.resize(hdr[2]);
    m.v.resize(hdr[2]);
    read_all(f, m.rp.data(), sizeof(int64_t) * m.rp.size());
    read_all(f, m.ci.data(), sizeof(int32_t) * m.ci.size());
    read_all(f, m.v.data(), sizeof(double) * m.v.size());
    if (m.rp[0] != 0 || m.rp[hdr[0]] != hdr[2]) fail(GEMSLR_ERR_ARG, "corrupt factor file (row pointers)");
}
gemslr_mat mat_view(const Csr &m) {
    gemslr_mat v;
    v.nrows = m.nrows;
    v.ncols = m.ncols;
    v.rowptr = m.rp.data();
    v.colind = m.ci.data();
    v.val = m.v.data();
    return v;
}
}  // namespace
extern "C" {

gemslr_status gemslr_save_factors(gemslr_handle h, const char *path) {
    return guard([&] {
        if (!h || !path) fail(GEMSLR_ERR_ARG, "NULL argument");
        if (h->host.cplx) fail(GEMSLR_ERR_UNSUPPORTED, "a complex handle cannot be saved");
        FilePtr f(fopen(path, "wb"));
        if (!f) fail(GEMSLR_ERR_ARG, std::string("cannot open ") + path + " for writing");
        const Hierarchy &H = h->host;
        write_all(f.get(), kFactorMagic, sizeof(kFactorMagic));
        const int64_t hdr[2] = {H.n, (int64_t)H.nlev};
        write_all(f.get(), hdr, sizeof(hdr));
        for (const HostLevel &hl : H.lev) {
            write_csr(f.get(), hl.L);
            write_csr(f.get(), hl.U);
            write_csr(f.get(), hl.E);
            write_csr(f.get(), hl.F);
            const int64_t k = hl.k;
            write_all(f.get(), &k, sizeof(k));
            write_all(f.get(), hl.W.data(), sizeof(double) * hl.W.size());
            write_all(f.get(), hl.H.data(), sizeof(double) * hl.H.size());
        }
        write_csr(f.get(), H.last.L);
        write_csr(f.get(), H.last.U);
        if (fflush(f.get()) != 0) fail(GEMSLR_ERR_ARG, "writing the factor file failed");
    });
}

gemslr_status gemslr_load_factors(const gemslr_csr *A, const gemslr_partition *part, const char *path,
                                  const gemslr_options *opt, gemslr_handle *out) {
    if (out) *out = nullptr;
    Hierarchy H;                               // file contents, kept alive for the views below
    std::vector<gemslr_level_factors> lf;
    gemslr_factors fac{};
    gemslr_status st = guard([&] {
        if (!A || !part || !path || !out) fail(GEMSLR_ERR_ARG, "NULL argument");
        FilePtr f(fopen(path, "rb"));
        if (!f) fail(GEMSLR_ERR_ARG, std::string("cannot open ") + path);
        char magic[8];
        read_all(f.get(), magic, sizeof(magic));
        if (std::memcmp(magic, kFactorMagic, sizeof(magic)) != 0) fail(GEMSLR_ERR_ARG, "not a GeMSLR factor file");
        int64_t hdr[2];
        read_all(f.get(), hdr, sizeof(hdr));
        if (hdr[0] != A->n) fail(GEMSLR_ERR_ARG, "factor file is for another matrix size");
        if (hdr[1] < 2 || hdr[1] > GEMSLR_MAX_LEVELS) fail(GEMSLR_ERR_ARG, "corrupt factor file (levels)");
        const int64_t lim = std::max<int64_t>(A->n, 1);
        H.lev.resize(hdr[1] - 1);
        lf.resize(H.lev.size());
        for (size_t l = 0; l < H.lev.size(); ++l) {
            HostLevel &hl = H.lev[l];
            read_csr(f.get(), hl.L, lim);
            read_csr(f.get(), hl.U, lim);
            read_csr(f.get(), hl.E, lim);
            read_csr(f.get(), hl.F, lim);
            int64_t k = 0;
            read_all(f.get(), &k, sizeof(k));
            if (k < 0 || k + 2 > kMaxRank) fail(GEMSLR_ERR_ARG, "corrupt factor file (rank)");
            hl.W.resize((size_t)hl.E.nrows * k);
            hl.H.resize((size_t)k * k);
            read_all(f.get(), hl.W.data(), sizeof(double) * hl.W.size());
            read_all(f.get(), hl.H.data(), sizeof(double) * hl.H.size());
            lf[l].L = mat_view(hl.L);
            lf[l].U = mat_view(hl.U);
            lf[l].E = mat_view(hl.E);
            lf[l].F = mat_view(hl.F);
            lf[l].k = (int32_t)k;
            lf[l].W = hl.W.data();
            lf[l].H = hl.H.data();
        }
        read_csr(f.get(), H.last.L, lim);
        read_csr(f.get(), H.last.U, lim);
        fac.nlev = (int32_t)hdr[1];
        fac.levels = lf.data();
        fac.last_L = mat_view(H.last.L);
        fac.last_U = mat_view(H.last.U);
    });
    if (st != GEMSLR_OK) return st;
    return gemslr_setup_from_factors(A, part, &fac, opt, out);
}

gemslr_status gemslr_apply(gemslr_handle h, const double *r_dev, double *z_dev, int32_t nrhs, void *stream) {
    return guard([&] {
        if (!h || nrhs < 0 || (nrhs > 0 && (!r_dev || !z_dev))) fail(GEMSLR_ERR_ARG, "invalid argument");
        if (r_dev == z_dev && nrhs > 0) fail(GEMSLR_ERR_ARG, "r and z must not alias");
        require_device(h);
        require_real(h);
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t n = h->host.n;
        ensure_krylov(h, 8);
        for (int c = 0; c < nrhs; ++c) {
            launch_gather(n, h->perm, r_dev + (size_t)c * n, h->bh, st);
            apply_perm(h, h->bh, h->xh, st);
            launch_scatter(n, h->perm, h->xh, z_dev + (size_t)c * n, st);
        }
        GEMSLR_CUDA(cudaGetLastError());
    });
}

gemslr_status gemslr_fgmres_solve(gemslr_handle h, const double *b_dev, double *x_dev, int32_t nrhs,
                                  const gemslr_solve_opts *opts, gemslr_solve_info *info, void *stream) {
    gemslr_status worst = GEMSLR_OK;
    gemslr_status st_ = guard([&] {
        if (!h || !opts || !info || nrhs < 0 || (nrhs > 0 && (!b_dev || !x_dev)))
            fail(GEMSLR_ERR_ARG, "invalid argument");
        require_device(h);
        require_real(h);
        if (opts->restart < 1 || opts->maxit < 1 || !(opts->rtol > 0) || opts->ortho < 0 || opts->ortho > 1)
            fail(GEMSLR_ERR_ARG, "invalid solve options");
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t n = h->host.n;
        const int m = opts->restart;
        ensure_krylov(h, m);
        for (int c = 0; c < nrhs; ++c) {
            auto t0 = std::chrono::steady_clock::now();
            gemslr_solve_info &inf = info[c];
            std::memset(&inf, 0, sizeof(inf));
            launch_gather(n, h->perm, b_dev + (size_t)c * n, h->bh, st);
            launch_norm2(n, h->bh, h->partial, h->counter, h->n2, h->red_grid, st);
            const double bn2 = read_scalar(h, h->n2, st);
            const double bnorm = std::sqrt(bn2);
            if (!std::isfinite(bnorm) || bnorm == 0.0) {
                launch_zero(n, h->xh, st);
                launch_scatter(n, h->perm, h->xh, x_dev + (size_t)c * n, st);
                if (bnorm == 0.0) {
                    inf.converged = 1;
                } else {
                    if (worst == GEMSLR_OK) worst = GEMSLR_ERR_NAN;
                    g_last_error = "right-hand side is not finite";
                }
                continue;
            }
            KrylovCtl cc{};
            cc.m = m;
            cc.givens = 1;
            cc.force_reorth = 0;
            cc.maxit = opts->maxit;
            cc.tol_abs = opts->rtol * bnorm;
            *h->ctl_host = cc;
            write_ctl(h, st);
            // GEMSLR_SOLVE_GRAPH=0 selects the host-driven loop (profilers cannot
            // see kernels inside conditional graph nodes)
            const char *env = std::getenv("GEMSLR_SOLVE_GRAPH");
            const bool allow_graph = !(env && env[0] == '0');
            const bool dcgs = opts->ortho == 0 && use_dcgs(h);
            const bool use_graph = allow_graph && !profile_enabled() && ensure_solve_graph(h, m, dcgs);
            if (use_graph) {
                GEMSLR_CUDA(cudaGraphLaunch(h->graph_exec, st));
                read_ctl(h, st);
                const KrylovCtl &k = *h->ctl_host;
                count_launch((int)(h->graph_k_top + (uint64_t)(k.restarts + 1) * h->graph_k_cycle +
                                   (uint64_t)k.iters * h->graph_k_step));
            } else {
                fgmres_host_loop(h, m, dcgs, st);
            }
            const KrylovCtl &k = *h->ctl_host;
            GEMSLR_CUDA(cudaMemcpyAsync(h->err_host, h->mixed ? h->d32.err : h->d64.err, 4, cudaMemcpyDeviceToHost, st));
            launch_scatter(n, h->perm, h->xh, x_dev + (size_t)c * n, st);
            GEMSLR_CUDA(cudaStreamSynchronize(st));
            inf.iters = k.iters;
            inf.restarts = k.restarts;
            inf.converged = k.converged ? 1 : 0;
            inf.reorth = k.nreorth;
            inf.rel_res_est = k.resid / bnorm;
            inf.rel_res_true = k.rnorm / bnorm;
            inf.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (h->err_host[0]) {
                GEMSLR_CUDA(cudaMemsetAsync(h->mixed ? h->d32.err : h->d64.err, 0, 4, st));
                fail(GEMSLR_ERR_TIMEOUT, "a bounded wait in the substitution kernel expired");
            }
            if (k.nonfinite) {
                if (worst == GEMSLR_OK) worst = GEMSLR_ERR_NAN;
                g_last_error = "FGMRES produced a non-finite value";
            } else if (!k.converged && worst == GEMSLR_OK) {
                worst = GEMSLR_ERR_NOT_CONVERGED;
                g_last_error = "FGMRES reached maxit";
            }
        }
    });
    return st_ != GEMSLR_OK ? st_ : worst;
}

gemslr_status gemslr_zapply(gemslr_handle h, const double *r_dev, double *z_dev, int32_t nrhs, void *stream) {
    return guard([&] {
        if (!h || nrhs < 0 || (nrhs > 0 && (!r_dev || !z_dev))) fail(GEMSLR_ERR_ARG, "invalid argument");
        if (r_dev == z_dev && nrhs > 0) fail(GEMSLR_ERR_ARG, "r and z must not alias");
        require_device(h);
        if (!h->host.cplx) fail(GEMSLR_ERR_ARG, "real handle: use gemslr_apply");
        z_apply(h->z, reinterpret_cast<const zc *>(r_dev), reinterpret_cast<zc *>(z_dev), nrhs,
                (cudaStream_t)stream);
    });
}

gemslr_status gemslr_zfgmres_solve(gemslr_handle h, const double *b_dev, double *x_dev, int32_t nrhs,
                                   const gemslr_solve_opts *opts, gemslr_solve_info *info, void *stream) {
    gemslr_status worst = GEMSLR_OK;
    gemslr_status st_ = guard([&] {
        if (!h || !opts || !info || nrhs < 0 || (nrhs > 0 && (!b_dev || !x_dev)))
            fail(GEMSLR_ERR_ARG, "invalid argument");
        require_device(h);
        if (!h->host.cplx) fail(GEMSLR_ERR_ARG, "real handle: use gemslr_fgmres_solve");
        if (opts->restart < 1 || opts->maxit < 1 || !(opts->rtol > 0)) fail(GEMSLR_ERR_ARG, "invalid solve options");
        const int64_t n = h->host.n;
        for (int c = 0; c < nrhs; ++c) {
            std::string msg;
            const gemslr_status s = z_solve(h->z, reinterpret_cast<const zc *>(b_dev) + (size_t)c * n,
                                            reinterpret_cast<zc *>(x_dev) + (size_t)c * n, *opts, info[c], msg,
                                            (cudaStream_t)stream);
            if (s != GEMSLR_OK && worst == GEMSLR_OK) {
                worst = s;
                g_last_error = msg;
            }
        }
    });
    return st_ != GEMSLR_OK ? st_ : worst;
}

gemslr_status gemslr_get_stats(gemslr_handle h, double *out, int32_t nout) {
    return guard([&] {
        if (!h || !out) fail(GEMSLR_ERR_ARG, "NULL argument");
        const Hierarchy &H = h->host;
        const int need = 8 + 6 * H.nlev;
        if (nout < need) fail(GEMSLR_ERR_ARG, "stats buffer too small");
        std::fill(out, out + nout, 0.0);
        int64_t nnzf = 0;
        for (auto &l : H.lev) nnzf += l.L.nnz() + l.U.nnz();
        nnzf += H.last.L.nnz() + H.last.U.nnz();
        out[0] = (double)H.n;
        out[1] = H.nlev;
        out[2] = (double)H.nclamp;
        out[3] = (double)H.Ahat.nnz();
        out[4] = (double)nnzf;
        // algorithmic bytes of one application (values, indices, vectors, W)
        const double sv = H.cplx ? 16.0 : (h->mixed ? 4.0 : 8.0), sw = H.cplx ? 16.0 : (h->mixed ? 2.0 : 8.0),
                     si = 4.0;
        double bytes = 0.0;
        for (auto &l : H.lev) {
            const double d = (double)(l.e - l.s), s = (double)(H.n - l.e);
            bytes += 2.0 * (l.L.nnz() + l.U.nnz()) * (sv + si);        // two substitutions
            bytes += (l.E.nnz() + l.F.nnz()) * (sv + si);
            bytes += 2.0 * s * l.k * sw;                               // W^T z and W u
            bytes += (8.0 * d + 6.0 * s) * sv;
        }
        bytes += (H.last.L.nnz() + H.last.U.nnz()) * (sv + si) + 2.0 * (H.n - H.last.s) * sv;
        bytes += 2.0 * H.n * (H.cplx ? 16.0 : 8.0);
        out[5] = bytes;
        out[6] = h->setup_ms;
        out[7] = (double)h->arena.bytes();
        for (int l = 0; l < H.nlev; ++l) {
            double *o = out + 8 + 6 * l;
            if (l + 1 < H.nlev) {
                const HostLevel &hl = H.lev[l];
                o[0] = (double)(hl.e - hl.s); o[1] = (double)(H.n - hl.e); o[2] = hl.k;
                o[3] = (double)(hl.L.nnz() + hl.U.nnz());
            } else {
                o[0] = (double)(H.n - H.last.s);
                o[3] = (double)(H.last.L.nnz() + H.last.U.nnz());
            }
            int wl = 0, wu = 0;
            if (H.cplx) z_wavefronts(h->z, l, wl, wu);
            else {
                const auto &dl = l + 1 < H.nlev ? h->d64.lev[l] : h->d64.last;
                wl = dl.nwf_L;
                wu = dl.nwf_U;
            }
            o[4] = wl;
            o[5] = wu;
        }
    });
}

void gemslr_destroy(gemslr_handle h) { delete h; }

uint64_t gemslr_kernel_launches(void) { return launches_total(); }

gemslr_status gemslr_selftest_wait(int64_t cycles) {
    return guard([&] {
        if (cycles <= 0) fail(GEMSLR_ERR_ARG, "cycles must be positive");
        int32_t *dev = nullptr;
        GEMSLR_CUDA(cudaMalloc(&dev, 2 * sizeof(int32_t)));
        int32_t host[2] = {0, 0};
        cudaError_t e = cudaMemset(dev, 0, 2 * sizeof(int32_t));
        if (e == cudaSuccess) {
            launch_wait_selftest((long long)cycles, dev, 0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(host, dev, sizeof(host), cudaMemcpyDeviceToHost);
        // the context must still be usable after the expired waits
        if (e == cudaSuccess) e = cudaMemset(dev, 0, 2 * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(dev);
        if (e != cudaSuccess) fail(GEMSLR_ERR_CUDA, cudaGetErrorString(e));
        if (host[0] != 1 || host[1] != 1) fail(GEMSLR_ERR_ARG, "a wait on an mbarrier that nothing completes returned");
        fail(GEMSLR_ERR_TIMEOUT, "bounded waits expired as expected (self-test)");
    });
}

void gemslr_profile_enable(int32_t on) { profile_enable(on != 0); }

void gemslr_profile_reset(void) { profile_reset(); }

int32_t gemslr_profile_read(char *names, size_t len, double *ms, int64_t *counts, int32_t maxn) {
    return profile_read(names, len, ms, counts, maxn);
}

}  // extern "C"

// ---- learned interface correction (not in the paper) ------------------------------------
namespace {

// Dense S_hat = C - E (LU)^{-1} F of level l (host, FP64) from the host factors.
std::vector<double> dense_schur(const Hierarchy &H, int l, std::vector<double> &diag) {
    const HostLevel &hl = H.lev[l];
    const int64_t d = hl.e - hl.s, S = H.n - hl.e;
    std::vector<double> X((size_t)d * S, 0.0), col(d);
    for (int64_t j = 0; j < S; ++j) {
        std::fill(col.begin(), col.end(), 0.0);
        for (int64_t i = 0; i < d; ++i)
            for (int64_t p = hl.F.rp[i]; p < hl.F.rp[i + 1]; ++p)
                if (hl.F.ci[p] == j) col[i] = hl.F.v[p];
        for (int64_t i = 0; i < d; ++i) {               // L y = col (unit lower)
            double s = col[i];
            for (int64_t p = hl.L.rp[i]; p < hl.L.rp[i + 1]; ++p) s -= hl.L.v[p] * col[hl.L.ci[p]];
            col[i] = s;
        }
        for (int64_t i = d - 1; i >= 0; --i) {          // U x = y
            double s = col[i], dg = 1.0;
            for (int64_t p = hl.U.rp[i]; p < hl.U.rp[i + 1]; ++p) {
                if (hl.U.ci[p] == i) dg = hl.U.v[p];
                else s -= hl.U.v[p] * col[hl.U.ci[p]];
            }
            col[i] = s / dg;
        }
        std::copy(col.begin(), col.end(), X.begin() + (size_t)j * d);
    }
    std::vector<double> Sh((size_t)S * S, 0.0);       // column-major
    for (int64_t i = 0; i < S; ++i)
        for (int64_t p = H.Ahat.rp[hl.e + i]; p < H.Ahat.rp[hl.e + i + 1]; ++p) {
            const int64_t c = H.Ahat.ci[p] - hl.e;
            if (c >= 0) Sh[(size_t)c * S + i] += H.Ahat.v[p];
        }
    for (int64_t i = 0; i < S; ++i)
        for (int64_t p = hl.E.rp[i]; p < hl.E.rp[i + 1]; ++p) {
            const int64_t k = hl.E.ci[p];
            const double ev = hl.E.v[p];
            for (int64_t j = 0; j < S; ++j) Sh[(size_t)j * S + i] -= ev * X[(size_t)j * d + k];
        }
    diag.resize(S);
    for (int64_t i = 0; i < S; ++i) diag[i] = Sh[(size_t)i * S + i];
    return Sh;
}

// Dense level-l* preconditioner M_S^{-1} = C~^{-1} (I + W H W^T), C~^{-1} the last-level block LU.
std::vector<double> dense_level_prec(const Hierarchy &H, int l) {
    const HostLevel &hl = H.lev[l];
    const HostLevel &la = H.last;
    const int64_t S = H.n - hl.e;
    if (l != (int)H.lev.size() - 1 || la.s != hl.e) fail(GEMSLR_ERR_UNSUPPORTED, "learned stage needs the deepest level");
    std::vector<double> P((size_t)S * S, 0.0), z(S), t;
    const int k = hl.k;
    for (int64_t j = 0; j < S; ++j) {
        std::fill(z.begin(), z.end(), 0.0);
        z[j] = 1.0;
        if (k > 0) {
            t.assign(k, 0.0);
            std::vector<double> u(k, 0.0);
            for (int c = 0; c < k; ++c) t[c] = hl.W[(size_t)c * S + j];
            for (int a = 0; a < k; ++a)
                for (int c = 0; c < k; ++c) u[a] += hl.H[a + (size_t)c * k] * t[c];
            for (int64_t i = 0; i < S; ++i)
                for (int c = 0; c < k; ++c) z[i] += hl.W[(size_t)c * S + i] * u[c];
        }
        for (int64_t i = 0; i < S; ++i) {
            double s = z[i];
            for (int64_t p = la.L.rp[i]; p < la.L.rp[i + 1]; ++p) s -= la.L.v[p] * z[la.L.ci[p]];
            z[i] = s;
        }
        for (int64_t i = S - 1; i >= 0; --i) {
            double s = z[i], dg = 1.0;
            for (int64_t p = la.U.rp[i]; p < la.U.rp[i + 1]; ++p) {
                if (la.U.ci[p] == i) dg = la.U.v[p];
                else s -= la.U.v[p] * z[la.U.ci[p]];
            }
            z[i] = s / dg;
        }
        std::copy(z.begin(), z.end(), P.begin() + (size_t)j * S);
    }
    return P;
}

// In-place inverse of a dense column-major matrix (Gauss-Jordan, partial pivoting).
void dense_inverse(std::vector<double> &A, int64_t n) {
    std::vector<double> Inv((size_t)n * n, 0.0);
    for (int64_t i = 0; i < n; ++i) Inv[(size_t)i * n + i] = 1.0;
    for (int64_t c = 0; c < n; ++c) {
        int64_t piv = c;
        for (int64_t i = c + 1; i < n; ++i)
            if (std::fabs(A[(size_t)c * n + i]) > std::fabs(A[(size_t)c * n + piv])) piv = i;
        if (A[(size_t)c * n + piv] == 0.0) fail(GEMSLR_ERR_NOT_CONVERGED, "S_hat is singular");
        if (piv != c)
            for (int64_t j = 0; j < n; ++j) {
                std::swap(A[(size_t)j * n + c], A[(size_t)j * n + piv]);
                std::swap(Inv[(size_t)j * n + c], Inv[(size_t)j * n + piv]);
            }
        const double inv = 1.0 / A[(size_t)c * n + c];
        for (int64_t j = 0; j < n; ++j) {
            A[(size_t)j * n + c] *= inv;
            Inv[(size_t)j * n + c] *= inv;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (i == c) continue;
            const double f = A[(size_t)c * n + i];
            if (f == 0.0) continue;
            for (int64_t j = 0; j < n; ++j) {
                A[(size_t)j * n + i] -= f * A[(size_t)j * n + c];
                Inv[(size_t)j * n + i] -= f * Inv[(size_t)j * n + c];
            }
        }
    }
    A.swap(Inv);
}

// Sites of level l*'s tail, neighbour table, weights (seeded He initialisation).
void learned_init(gemslr_ctx *h, LearnedHost &Lh, const int32_t *coords, int channels, uint64_t seed) {
    const Hierarchy &H = h->host;
    if (H.lev.empty()) fail(GEMSLR_ERR_UNSUPPORTED, "learned stage needs a Schur level");
    if (channels < 1 || channels > 32) fail(GEMSLR_ERR_ARG, "channels must be in 1..32");
    Lh.lstar = (int)H.lev.size() - 1;
    Lh.e = H.lev[Lh.lstar].e;
    const int64_t S = H.n - Lh.e;
    NetDev &net = Lh.net;
    net.S = (int)S;
    net.C = channels;
    const int dims[5] = {1, channels, channels, channels, 1};
    std::unordered_map<uint64_t, int32_t> where;
    auto key = [](int64_t x, int64_t y, int64_t z) {
        return ((uint64_t)(x + 1) << 42) | ((uint64_t)(y + 1) << 21) | (uint64_t)(z + 1);
    };
    std::vector<int64_t> cx(S), cy(S), cz(S);
    for (int64_t s = 0; s < S; ++s) {
        const int64_t o = H.perm[Lh.e + s];
        cx[s] = coords[3 * o];
        cy[s] = coords[3 * o + 1];
        cz[s] = coords[3 * o + 2];
        where[key(cx[s], cy[s], cz[s])] = (int32_t)s;
    }
    std::vector<int32_t> nbr((size_t)S * 27, -1);
    for (int64_t s = 0; s < S; ++s)
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    auto it = where.find(key(cx[s] + dx, cy[s] + dy, cz[s] + dz));
                    nbr[(size_t)s * 27 + t] = it == where.end() ? -1 : it->second;
                }
    Arena &a = h->arena;
    net.nbr = a.upload(nbr);
    net.nparams = 0;
    for (int l = 0; l < kNetLayers; ++l) {
        net.cin[l] = dims[l];
        net.cout[l] = dims[l + 1];
        const int64_t nw = 27LL * dims[l] * dims[l + 1];
        std::vector<double> u = splitmix_uniform01(seed * 100 + (uint64_t)l, nw);
        const double bound = std::sqrt(6.0 / (27.0 * dims[l])) * (l < 3 ? 1.0 : 0.1);
        std::vector<float> w(nw);
        for (int64_t i = 0; i < nw; ++i) w[i] = (float)((2.0 * u[i] - 1.0) * bound);
        net.W[l] = a.upload(w);
        net.b[l] = (float *)a.alloc(4 * dims[l + 1]);
        GEMSLR_CUDA(cudaMemset(net.b[l], 0, 4 * dims[l + 1]));
        net.Wb[l] = (__nv_bfloat16 *)a.alloc(2 * nw);
        net.gW[l] = (float *)a.alloc(4 * nw);
        net.gb[l] = (float *)a.alloc(4 * dims[l + 1]);
        net.mW[l] = (float *)a.alloc(4 * nw);
        net.vW[l] = (float *)a.alloc(4 * nw);
        net.mb[l] = (float *)a.alloc(4 * dims[l + 1]);
        net.vb[l] = (float *)a.alloc(4 * dims[l + 1]);
        GEMSLR_CUDA(cudaMemset(net.mW[l], 0, 4 * nw));
        GEMSLR_CUDA(cudaMemset(net.vW[l], 0, 4 * nw));
        GEMSLR_CUDA(cudaMemset(net.mb[l], 0, 4 * dims[l + 1]));
        GEMSLR_CUDA(cudaMemset(net.vb[l], 0, 4 * dims[l + 1]));
        net.nparams += nw + dims[l + 1];
    }
    net.adam_t = 0;
    net_kernels_init();
    net_sync_bf16(net, nullptr);
    // in-apply buffers for both precisions
    const HostLevel &hl = H.lev[Lh.lstar];
    Csr C = submatrix(H.Ahat, hl.e, H.n, hl.e, H.n);
    auto setup_stage = [&](auto &st, auto tag) {
        using VT = decltype(tag);
        st.net = &Lh.net;
        st.zsave = (VT *)a.alloc(sizeof(VT) * S);
        st.work2 = (VT *)a.alloc(sizeof(VT) * H.n);
        st.zeros = h->zeros;
        st.C_rp = a.upload(C.rp);
        st.C_ci = a.upload(C.ci);
        st.C_v = a.upload(convert<VT>(C.v));
        st.act0 = (float *)a.alloc(4 * S);
        st.act1 = (float *)a.alloc(4 * S * channels);
        st.act2 = (float *)a.alloc(4 * S * channels);
        st.rnorm = (float *)a.alloc(16);
    };
    setup_stage(Lh.st64, double(0));
    setup_stage(Lh.st32, float(0));
    h->d64.learned = &Lh.st64;
    if (h->mixed) h->d32.learned = &Lh.st32;
}

// Batch buffers of one training / gradient pass.
struct PassBufs {
    int B = 0;
    float *zs[4], *hs[3], *g0, *g1, *dout, *loss, *part;
    int nchunk = 0;
};

PassBufs pass_bufs(gemslr_ctx *h, const NetDev &net, int B) {
    PassBufs p;
    p.B = B;
    Arena &a = h->arena;
    const int64_t SC = (int64_t)net.S * net.C * B;
    for (int l = 0; l < 4; ++l) p.zs[l] = (float *)a.alloc(4 * (l < 3 ? SC : (int64_t)net.S * B));
    for (int l = 0; l < 3; ++l) p.hs[l] = (float *)a.alloc(4 * SC);
    p.g0 = (float *)a.alloc(4 * SC);
    p.g1 = (float *)a.alloc(4 * SC);
    p.dout = (float *)a.alloc(4 * (int64_t)net.S * B);
    p.loss = (float *)a.alloc(4 * B);
    p.nchunk = 64;
    p.part = (float *)a.alloc(4 * (int64_t)p.nchunk * 27 * net.C * net.C);
    return p;
}

// Forward, loss and backward on one batch (x0: B x S inputs, y: targets).
void train_pass(NetDev &net, PassBufs &pb, const float *x0, const float *y, cudaStream_t st) {
    net_forward(net, pb.B, x0, pb.zs, pb.hs, st);
    launch_loss(net.S, pb.B, pb.zs[3], y, pb.dout, pb.loss, st);
    net_backward(net, pb.B, x0, pb.zs, pb.hs, pb.dout, pb.g0, pb.g1, pb.part, pb.nchunk, st);
}

}  // namespace

extern "C" {

gemslr_status gemslr_learned_train(gemslr_handle h, const int32_t *coords, const gemslr_learned_opts *o,
                                   double *loss_history) {
    return guard([&] {
        if (!h || !coords || !o) fail(GEMSLR_ERR_ARG, "NULL argument");
        require_real(h);
        if (h->d64.inner.k > 0 || h->d32.inner.k > 0)
            fail(GEMSLR_ERR_ARG, "inner steps and the learned stage are exclusive");
        if (o->npairs < 1 || o->epochs < 0 || o->batch < 1 || !(o->lr > 0)) fail(GEMSLR_ERR_ARG, "invalid learned options");
        if (!h->learned) h->learned = new LearnedHost();
        LearnedHost &Lh = *h->learned;
        learned_init(h, Lh, coords, o->channels, o->seed);
        NetDev &net = Lh.net;
        const Hierarchy &H = h->host;
        const int64_t S = net.S;
        cudaStream_t st = nullptr;
        // training pairs (rho, S_hat^{-1} rho) from the method's own level-l* application
        std::vector<double> diag;
        std::vector<double> Sh = dense_schur(H, Lh.lstar, diag);
        std::vector<double> P = dense_level_prec(H, Lh.lstar);
        double dmean = 0.0;
        for (double v : diag) dmean += std::fabs(v);
        net.dscale = S > 0 ? dmean / S : 1.0;
        Arena &a = h->arena;
        double *dS = a.upload(Sh), *dP = a.upload(P);
        double *dR = (double *)a.alloc(8 * (size_t)S * S);
        launch_dgemm((int)S, (int)S, (int)S, dS, dP, dR, st);                    // S_hat P
        std::vector<double> R((size_t)S * S);
        GEMSLR_CUDA(cudaMemcpy(R.data(), dR, 8 * R.size(), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < R.size(); ++i) R[i] = -R[i];
        for (int64_t i = 0; i < S; ++i) R[(size_t)i * S + i] += 1.0;          // I - S_hat P
        GEMSLR_CUDA(cudaMemcpy(dR, R.data(), 8 * R.size(), cudaMemcpyHostToDevice));
        dense_inverse(Sh, S);
        double *dSi = a.upload(Sh);
        const int64_t N = o->npairs;
        double *Z = (double *)a.alloc(8 * (size_t)S * N), *RHO = (double *)a.alloc(8 * (size_t)S * N),
               *T = (double *)a.alloc(8 * (size_t)S * N);
        launch_uniform(o->seed ^ 0x5eedULL, (int64_t)S * N, Z, st);
        launch_dgemm((int)S, (int)N, (int)S, dR, Z, RHO, st);
        launch_dgemm((int)S, (int)N, (int)S, dSi, RHO, T, st);
        float *X = (float *)a.alloc(4 * (size_t)S * N), *Y = (float *)a.alloc(4 * (size_t)S * N);
        launch_scale_pairs((int)S, (int)N, RHO, T, net.dscale, X, Y, st);
        // training: Adam, sequential batches
        const int B = std::min<int64_t>(o->batch, N);
        PassBufs pb = pass_bufs(h, net, B);
        std::vector<float> lossb(B);
        for (int ep = 0; ep < o->epochs; ++ep) {
            double acc = 0.0;
            int64_t cnt = 0;
            for (int64_t i0 = 0; i0 + B <= N; i0 += B) {
                train_pass(net, pb, X + i0 * S, Y + i0 * S, st);
                net_adam(net, (float)o->lr, st);
                GEMSLR_CUDA(cudaMemcpyAsync(lossb.data(), pb.loss, 4 * B, cudaMemcpyDeviceToHost, st));
                GEMSLR_CUDA(cudaStreamSynchronize(st));
                for (float v : lossb) acc += v;
                cnt += B;
            }
            if (loss_history) loss_history[ep] = cnt ? acc / cnt : 0.0;
        }
        GEMSLR_CUDA(cudaDeviceSynchronize());
        Lh.st64.enabled = Lh.st32.enabled = true;
        if (h->graph_exec) {                 // the captured solve must include the new stage
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
            cudaGraphDestroy(h->graph);
            h->graph = nullptr;
        }
    });
}

gemslr_status gemslr_set_inner_steps(gemslr_handle h, int32_t steps) {
    return guard([&] {
        if (!h || steps < 0 || steps > kMaxInner) fail(GEMSLR_ERR_ARG, "inner steps must be in [0, 8]");
        require_real(h);
        if (steps > 0 && h->host.lev.empty()) fail(GEMSLR_ERR_ARG, "inner steps need a Schur level");
        const bool learned = (h->d64.learned && h->d64.learned->enabled) || (h->d32.learned && h->d32.learned->enabled);
        if (steps > 0 && learned) fail(GEMSLR_ERR_ARG, "inner steps and the learned stage are exclusive");
        if (h->mixed) setup_inner<float, __nv_bfloat16>(h->host, h->arena, h->d32, steps, sm_count());
        else setup_inner<double, double>(h->host, h->arena, h->d64, steps, sm_count());
        if (h->graph_exec) {                 // the captured solve depends on M^{-1}: rebuild on next use
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
            cudaGraphDestroy(h->graph);
            h->graph = nullptr;
        }
        GEMSLR_CUDA(cudaDeviceSynchronize());
    });
}

gemslr_status gemslr_learned_enable(gemslr_handle h, int32_t on) {
    return guard([&] {
        if (!h || !h->learned) fail(GEMSLR_ERR_ARG, "no learned stage on this handle");
        if (on && (h->d64.inner.k > 0 || h->d32.inner.k > 0))
            fail(GEMSLR_ERR_ARG, "inner steps and the learned stage are exclusive");
        h->learned->st64.enabled = h->learned->st32.enabled = on != 0;
        if (h->graph_exec) {                 // the captured solve depends on the stage: rebuild on next use
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
            cudaGraphDestroy(h->graph);
            h->graph = nullptr;
        }
    });
}

gemslr_status gemslr_learned_info(gemslr_handle h, double *out) {
    return guard([&] {
        if (!h || !h->learned || !out) fail(GEMSLR_ERR_ARG, "no learned stage on this handle");
        const NetDev &net = h->learned->net;
        out[0] = net.S;
        out[1] = net.C;
        out[2] = net.dscale;
        out[3] = (double)net.nparams;
    });
}

gemslr_status gemslr_learned_params(gemslr_handle h, int32_t get, double *params, int64_t n) {
    return guard([&] {
        if (!h || !h->learned || !params) fail(GEMSLR_ERR_ARG, "no learned stage on this handle");
        NetDev &net = h->learned->net;
        if (n != net.nparams) fail(GEMSLR_ERR_ARG, "parameter count mismatch");
        int64_t off = 0;
        for (int l = 0; l < kNetLayers; ++l) {
            const int64_t nw = 27LL * net.cin[l] * net.cout[l], nb = net.cout[l];
            std::vector<float> w(nw), b(nb);
            if (get) {
                GEMSLR_CUDA(cudaMemcpy(w.data(), net.W[l], 4 * nw, cudaMemcpyDeviceToHost));
                GEMSLR_CUDA(cudaMemcpy(b.data(), net.b[l], 4 * nb, cudaMemcpyDeviceToHost));
                for (int64_t i = 0; i < nw; ++i) params[off + i] = w[i];
                for (int64_t i = 0; i < nb; ++i) params[off + nw + i] = b[i];
            } else {
                for (int64_t i = 0; i < nw; ++i) w[i] = (float)params[off + i];
                for (int64_t i = 0; i < nb; ++i) b[i] = (float)params[off + nw + i];
                GEMSLR_CUDA(cudaMemcpy(net.W[l], w.data(), 4 * nw, cudaMemcpyHostToDevice));
                GEMSLR_CUDA(cudaMemcpy(net.b[l], b.data(), 4 * nb, cudaMemcpyHostToDevice));
            }
            off += nw + nb;
        }
        if (!get) {
            net_sync_bf16(net, nullptr);
            GEMSLR_CUDA(cudaDeviceSynchronize());
        }
    });
}

gemslr_status gemslr_learned_loss_grad(gemslr_handle h, int32_t nb, const double *x, const double *y, double *loss,
                                       double *grad) {
    return guard([&] {
        if (!h || !h->learned || nb < 1 || !x || !y || !loss || !grad) fail(GEMSLR_ERR_ARG, "invalid argument");
        NetDev &net = h->learned->net;
        const int64_t S = net.S;
        std::vector<float> xf((size_t)nb * S), yf((size_t)nb * S);
        for (size_t i = 0; i < xf.size(); ++i) { xf[i] = (float)x[i]; yf[i] = (float)y[i]; }
        Arena tmp;
        float *dx = tmp.upload(xf), *dy = tmp.upload(yf);
        PassBufs pb = pass_bufs(h, net, nb);
        train_pass(net, pb, dx, dy, nullptr);
        std::vector<float> l(nb);
        GEMSLR_CUDA(cudaMemcpy(l.data(), pb.loss, 4 * nb, cudaMemcpyDeviceToHost));
        double acc = 0.0;
        for (float v : l) acc += v;
        *loss = acc / nb;
        int64_t off = 0;
        for (int lyr = 0; lyr < kNetLayers; ++lyr) {
            const int64_t nw = 27LL * net.cin[lyr] * net.cout[lyr], nbias = net.cout[lyr];
            std::vector<float> gw(nw), gbv(nbias);
            GEMSLR_CUDA(cudaMemcpy(gw.data(), net.gW[lyr], 4 * nw, cudaMemcpyDeviceToHost));
            GEMSLR_CUDA(cudaMemcpy(gbv.data(), net.gb[lyr], 4 * nbias, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < nw; ++i) grad[off + i] = gw[i];
            for (int64_t i = 0; i < nbias; ++i) grad[off + nw + i] = gbv[i];
            off += nw + nbias;
        }
    });
}

}  // extern "C"

// ---- allocation-free application -------------------------------------------------------
// Some callers cannot allocate device memory at the point where they need
// M^{-1}: code that runs while a stream is being captured into a CUDA graph
// (cudaMalloc is not allowed there in the global capture mode), callers that
// hand all device memory to their own pool or allocator and forbid other
// allocations, and latency-bound loops that must not hit the allocator's
// synchronisation.  gemslr_apply may allocate its permutation buffers on
// first use; gemslr_apply_static never does: it keeps the permuted copies of
// r and z in a fixed file-scope device array.
namespace {
constexpr int64_t kStaticRows = int64_t(1) << 21;                  // 2,097,152 rows per vector
__device__ __align__(256) double g_static_scratch[2 * kStaticRows];  // 32 MiB, held by every GPU that loads the library
constexpr int kMaxDevices = 64;
double *g_static_addr[kMaxDevices] = {};
std::mutex g_static_mu;
}  // namespace

extern "C" gemslr_status gemslr_apply_static(gemslr_handle h, const double *r_dev, double *z_dev, void *stream) {
    return guard([&] {
        if (!h || !r_dev || !z_dev) fail(GEMSLR_ERR_ARG, "NULL argument");
        if (r_dev == z_dev) fail(GEMSLR_ERR_ARG, "r and z must not alias");
        const int64_t n = h->host.n;
        if (n > kStaticRows)
            fail(GEMSLR_ERR_ARG, "n = " + std::to_string(n) + " exceeds the static scratch capacity of " +
                                     std::to_string(kStaticRows) + " rows; use gemslr_apply");
        require_device(h);
        require_real(h);
        const int dev = h->dev;
        if (dev < 0 || dev >= kMaxDevices) fail(GEMSLR_ERR_ARG, "device index out of range");
        double *base = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_static_mu);
            if (!g_static_addr[dev]) {      // once per device, with that device current
                void *p = nullptr;
                const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
                if (e != cudaSuccess) fail(GEMSLR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                g_static_addr[dev] = static_cast<double *>(p);
            }
            base = g_static_addr[dev];
        }
        cudaStream_t st = (cudaStream_t)stream;
        double *pin = base, *pout = base + kStaticRows;
        launch_gather(n, h->perm, r_dev, pin, st);
        apply_perm(h, pin, pout, st);
        launch_scatter(n, h->perm, pout, z_dev, st);
        GEMSLR_CUDA(cudaGetLastError());
    });
}
