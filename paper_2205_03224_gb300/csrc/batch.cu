// Batched GeMSLR-FGMRES: many independent systems with up to kBatchRhs
// right-hand sides each.  Setup (Alg. 1) runs per system; the solve phase
// launches every stage of M^{-1} (Alg. 2) once over all systems and runs
// FGMRES (Sec. 4.1) for every (system, rhs) pair in lock step inside one CUDA
// graph with conditional WHILE nodes.  The preconditioner is FP32 (W in BF16
// with FP32 accumulation); the Krylov vectors, least-squares problems and
// residuals are FP64.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <exception>
#include <memory>
#include <thread>

#include "batch.cuh"
#include "device.h"

namespace gemslr {
void launch_btrsv(const BatchLevel &lv, int mode, int rpc, size_t smem_bytes, const double *in, float *work,
                  double *out_final, float *scratch, cudaStream_t st);
void set_btrsv_smem_limit(int bytes);
void launch_bcouple(const BatchLevel &lv, const double *in, float *work, cudaStream_t st);
void launch_blowrank(const BatchLevel &lv, float *work, cudaStream_t st);
void launch_bspmv(int64_t nrows, const int64_t *rp, const int32_t *ci, const double *v, const double *x,
                  const double *b, double *y, double *zcol, const int32_t *jp, int64_t ld, cudaStream_t st,
                  const int32_t *sys_of = nullptr, const int32_t *live = nullptr);
void launch_bgs(int pass, const BatchSegs &S, const BatchKrylov &K, double *V, int64_t ldv, double *w,
                cudaStream_t st);
void launch_bgs_subnorm(const BatchSegs &S, const BatchKrylov &K, double *V, int64_t ldv, double *w,
                        cudaStream_t st);
void launch_bgs_final(const BatchSegs &S, const BatchKrylov &K, double *V, int64_t ldv, const double *w, double *vin,
                      cudaStream_t st);
void launch_bnorm2(const BatchSegs &S, double *partial, const double *x, double *out, cudaStream_t st);
void launch_binit(const BatchKrylov &K, double rtol, int maxit, cudaStream_t st);
void launch_bcycle_start(const BatchKrylov &K, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st);
void launch_bscale(const BatchSegs &S, const BatchKrylov &K, const double *r, double *V, double *vin, cudaStream_t st);
void launch_bstep_end(const BatchKrylov &K, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st);
void launch_blsq(const BatchKrylov &K, cudaStream_t st);
void launch_bupdate_x(const BatchSegs &S, const BatchKrylov &K, const double *Z, int64_t ldz, double *x,
                      cudaStream_t st);
void launch_bcycle_end(const BatchKrylov &K, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st);
void launch_bgather(int64_t nrows, const int32_t *sys_of, const int64_t *perm_g, const int64_t *usr_off,
                    const int64_t *nsz, int nrhs, const double *src, double *dst, cudaStream_t st);
void launch_bscatter(int64_t nrows, const int32_t *sys_of, const int64_t *perm_g, const int64_t *usr_off,
                     const int64_t *nsz, int nrhs, const double *src, double *dst, cudaStream_t st);
cudaGraph_t capture_while_node(cudaStream_t cs, cudaGraphConditionalHandle handle);
}  // namespace gemslr

using namespace gemslr;

struct BLevelHost {          // device level plus what the launcher needs
    BatchLevel v{};
    int rpc = 0;              // right-hand sides per substitution CTA (0: vector in global memory)
    size_t smem_bytes = 0;
    int64_t rows = 0;         // rows of the level's blocks, all systems
    int64_t l_bytes = 0, u_bytes = 0;   // stored L and U chunks
    int64_t f_nnz = 0;        // nonzeros of F
};

struct gemslr_batch_ctx {
    int nsys = 0, nlev = 0;
    int dev = 0;                            // the device the batch was set up on
    int64_t N = 0;                          // batch rows
    std::vector<Hierarchy> sys;
    std::vector<int64_t> base;              // nsys + 1
    Arena arena;
    std::vector<BLevelHost> lev;            // Schur levels then the last level (index nlev-1)
    float *work = nullptr, *scratch = nullptr;
    int32_t *err = nullptr;
    // Krylov
    int64_t *A_rp = nullptr;
    int32_t *A_ci = nullptr;
    double *A_v = nullptr;
    int32_t *sys_of = nullptr;
    int64_t *perm_g = nullptr, *nsz = nullptr, *usr_off = nullptr;
    BatchSegs S{};
    BatchKrylov K{};
    int m_alloc = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *x = nullptr, *b = nullptr, *r = nullptr, *vin = nullptr,
           *zout = nullptr;
    // graphs
    cudaStream_t cap = nullptr;
    cudaGraphExec_t apply_exec = nullptr, solve_exec = nullptr;
    cudaGraph_t apply_graph = nullptr, solve_graph = nullptr;
    int solve_m = 0;
    uint64_t k_apply = 0, k_top = 0, k_cycle = 0, k_step = 0;
    // autotuned work-list sizes
    int rows_couple = 128, rows_krylov = kKrylovRows;
    double setup_ms = 0.0, tune_ms = 0.0;
    std::vector<int32_t> host_ints;
    ~gemslr_batch_ctx() {
        if (apply_exec) cudaGraphExecDestroy(apply_exec);
        if (apply_graph) cudaGraphDestroy(apply_graph);
        if (solve_exec) cudaGraphExecDestroy(solve_exec);
        if (solve_graph) cudaGraphDestroy(solve_graph);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

thread_local std::string g_batch_error;

gemslr_status bguard(const std::function<void()> &fn) {
    try {
        fn();
        return GEMSLR_OK;
    } catch (const Error &e) {
        g_batch_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_batch_error = "host allocation failed";
        return GEMSLR_ERR_NOMEM;
    } catch (const std::exception &e) {
        g_batch_error = e.what();
        return GEMSLR_ERR_ARG;
    }
}

int dev_smem_optin() {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return b;
}

// Start row of level l of system s inside the batch, its blocks, E/F/W.
void build_batch_level(gemslr_batch_ctx *B, int l, bool last, int rows_cta, BLevelHost &out) {
    ChunkHost<float> ch;
    std::vector<int64_t> blk_r0, blk_f0, F_rp{0}, E_rp{0}, seg_r0, seg_len, seg_e0, seg_w0, seg_h0;
    std::vector<int32_t> blk_nr, blk_sys, F_ci, E_ci, seg_k, cta_seg, seg_cta0{0};
    std::vector<int64_t> cta_i0;
    std::vector<float> F_v, E_v, H;
    std::vector<__nv_bfloat16> W;
    int64_t frows = 0, maxrows = 0;
    for (int s = 0; s < B->nsys; ++s) {
        const Hierarchy &h = B->sys[s];
        const HostLevel &hl = last ? h.last : h.lev[l];
        const int64_t bs = B->base[s];
        ChunkHost<float> cs;
        build_chunks<float>(hl.L, hl.U, hl.bp, cs, kBatchChunkRows, 1, kStageBytes);
        // append chunk data with offsets shifted
        const int64_t doff = (int64_t)ch.data.size();
        const int64_t coff = (int64_t)ch.off.size() - 1;
        ch.data.insert(ch.data.end(), cs.data.begin(), cs.data.end());
        for (size_t q = 1; q < cs.off.size(); ++q) ch.off.push_back(cs.off[q] + doff);
        // cs.data may carry a 16-byte filler when it has no chunks; keep offsets consistent
        if (cs.off.size() == 1 && !cs.data.empty()) { /* filler bytes are never referenced */ }
        for (size_t j = 0; j + 1 < hl.bp.size(); ++j) {
            blk_r0.push_back(bs + hl.s + hl.bp[j]);
            blk_nr.push_back((int32_t)(hl.bp[j + 1] - hl.bp[j]));
            blk_sys.push_back(s);
            blk_f0.push_back(frows + hl.bp[j]);
            maxrows = std::max(maxrows, hl.bp[j + 1] - hl.bp[j]);
            ch.blk_chunk.push_back((int32_t)(coff + cs.blk_chunk[j + 1]));
        }
        if (!last) {
            for (int64_t i = 0; i < hl.F.nrows; ++i) {
                for (int64_t p = hl.F.rp[i]; p < hl.F.rp[i + 1]; ++p) {
                    F_ci.push_back((int32_t)(bs + hl.e + hl.F.ci[p]));
                    F_v.push_back((float)hl.F.v[p]);
                }
                F_rp.push_back((int64_t)F_ci.size());
            }
            const int64_t len = h.n - hl.e;
            seg_r0.push_back(bs + hl.e);
            seg_len.push_back(len);
            seg_e0.push_back((int64_t)E_rp.size() - 1);
            for (int64_t i = 0; i < hl.E.nrows; ++i) {
                for (int64_t p = hl.E.rp[i]; p < hl.E.rp[i + 1]; ++p) {
                    E_ci.push_back((int32_t)(bs + hl.s + hl.E.ci[p]));
                    E_v.push_back((float)hl.E.v[p]);
                }
                E_rp.push_back((int64_t)E_ci.size());
            }
            if (hl.k > kBatchMaxRank) fail(GEMSLR_ERR_ARG, "batched rank above 64");
            seg_k.push_back(hl.k);
            seg_w0.push_back((int64_t)W.size());
            seg_h0.push_back((int64_t)H.size());
            for (double v : hl.W) W.push_back(__float2bfloat16_rn((float)v));
            for (double v : hl.H) H.push_back((float)v);
            for (int64_t i0 = 0; i0 < len; i0 += rows_cta) {
                cta_seg.push_back(s);
                cta_i0.push_back(i0);
            }
            seg_cta0.push_back((int32_t)cta_seg.size());
        }
        frows += hl.e - hl.s;
    }
    out.rows = out.l_bytes = out.u_bytes = 0;    // the level may be rebuilt (autotuning)
    for (size_t c = 0; c + 1 < ch.off.size(); ++c) {
        int32_t upper = 0;
        std::memcpy(&upper, ch.data.data() + ch.off[c] + 8, 4);
        (upper ? out.u_bytes : out.l_bytes) += ch.off[c + 1] - ch.off[c];
    }
    for (int32_t nr : blk_nr) out.rows += nr;
    out.f_nnz = (int64_t)F_ci.size();
    if (ch.data.empty()) ch.data.resize(16, 0);
    Arena &a = B->arena;
    BatchLevel &v = out.v;
    v.nblk = (int32_t)blk_r0.size();
    // CTAs are dispatched in index order and a block's time grows with its
    // chunk count (one consumer barrier per chunk): the blocks with the most
    // chunks go first, so that no long block starts in the last wave
    std::vector<int32_t> order(v.nblk);
    for (int32_t j = 0; j < v.nblk; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return ch.blk_chunk[x + 1] - ch.blk_chunk[x] > ch.blk_chunk[y + 1] - ch.blk_chunk[y];
    });
    v.order = a.upload(order);
    v.blk_sys = a.upload(blk_sys);
    v.live = nullptr;
    v.final_up = (!last && l == 0) ? 1 : 0;
    v.blk_r0 = a.upload(blk_r0);
    v.blk_nr = a.upload(blk_nr);
    v.blk_f0 = a.upload(blk_f0);
    v.C.data = a.upload(ch.data);
    v.C.off = a.upload(ch.off);
    v.C.blk_chunk = a.upload(ch.blk_chunk);
    v.err = B->err;
    const int optin = dev_smem_optin();
    // the most right-hand sides per CTA whose block vectors fit in shared
    // memory; a split (fewer than kBatchRhs) multiplies the CTAs, and is taken
    // only while they all fit on the GPU at once: otherwise the CTAs would run
    // in many waves, slower than one wave with the vectors in global memory
    out.rpc = 0;
    out.smem_bytes = 0;
    for (int rpc = kBatchRhs; rpc >= 1; rpc /= 2) {
        const size_t bytes = (size_t)kRingBytes + (size_t)maxrows * rpc * sizeof(float);
        if (bytes <= (size_t)optin) {
            out.rpc = rpc;
            out.smem_bytes = bytes;
            break;
        }
    }
    if (out.rpc > 0 && out.rpc < kBatchRhs) {
        int dev = 0, sms = 1, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int64_t resident = (int64_t)sms * std::max<int64_t>(1, per_sm / (int64_t)out.smem_bytes);
        if ((int64_t)v.nblk * (kBatchRhs / out.rpc) > resident) {
            out.rpc = 0;
            out.smem_bytes = 0;
        }
    }
    if (!last) {
        v.F_rp = a.upload(F_rp);
        v.F_ci = a.upload(F_ci);
        v.F_v = a.upload(F_v);
        v.nseg = B->nsys;
        v.seg_r0 = a.upload(seg_r0);
        v.seg_len = a.upload(seg_len);
        v.seg_e0 = a.upload(seg_e0);
        v.E_rp = a.upload(E_rp);
        v.E_ci = a.upload(E_ci);
        v.E_v = a.upload(E_v);
        v.seg_w0 = a.upload(seg_w0);
        v.seg_k = a.upload(seg_k);
        v.seg_h0 = a.upload(seg_h0);
        v.W = a.upload(W);
        v.H = a.upload(H);
        v.ncta = (int32_t)cta_seg.size();
        v.rows_cta = rows_cta;
        v.cta_seg = a.upload(cta_seg);
        v.cta_i0 = a.upload(cta_i0);
        v.seg_cta0 = a.upload(seg_cta0);
        v.seg_counter = (unsigned *)a.alloc(sizeof(unsigned) * std::max(1, B->nsys));
        GEMSLR_CUDA(cudaMemset(v.seg_counter, 0, sizeof(unsigned) * std::max(1, B->nsys)));
        v.partial = (float *)a.alloc(sizeof(float) * std::max<int64_t>(1, v.ncta) * kBatchMaxRank * kBatchRhs);
        v.u = (float *)a.alloc(sizeof(float) * std::max(1, B->nsys) * kBatchMaxRank * kBatchRhs);
    }
}

// M^{-1} on the batch layout: in (FP64) -> out (FP64), every stage one launch.
// live (nsys flags, or nullptr): systems whose flag is 0 are skipped.
void batch_apply_layout(gemslr_batch_ctx *B, const double *in, double *out, cudaStream_t st,
                        const int32_t *live = nullptr) {
    const int ns = B->nlev - 1;
    auto lv = [&](int l) {
        BatchLevel v = B->lev[l].v;
        v.live = live;
        return v;
    };
    for (int l = 0; l < ns; ++l) {
        const double *src = l == 0 ? in : nullptr;
        launch_btrsv(lv(l), 0, B->lev[l].rpc, B->lev[l].smem_bytes, src, B->work, nullptr, B->scratch, st);
        launch_bcouple(lv(l), src, B->work, st);
        launch_blowrank(lv(l), B->work, st);
    }
    const BLevelHost &la = B->lev[ns];
    launch_btrsv(lv(ns), 0, la.rpc, la.smem_bytes, ns == 0 ? in : nullptr, B->work, out, B->scratch, st);
    for (int l = ns - 1; l >= 0; --l)
        launch_btrsv(lv(l), 1, B->lev[l].rpc, B->lev[l].smem_bytes, nullptr, B->work, out, B->scratch, st);
}

void build_segments(gemslr_batch_ctx *B, int rows) {
    std::vector<int32_t> cta_sys, sys_cta0{0};
    std::vector<int64_t> cta_r0, cta_r1;
    for (int s = 0; s < B->nsys; ++s) {
        for (int64_t g = B->base[s]; g < B->base[s + 1]; g += rows) {
            cta_sys.push_back(s);
            cta_r0.push_back(g);
            cta_r1.push_back(std::min(g + rows, B->base[s + 1]));
        }
        sys_cta0.push_back((int32_t)cta_sys.size());
    }
    Arena &a = B->arena;
    B->S.nsys = B->nsys;
    B->S.sys_r0 = a.upload(B->base);
    B->S.ncta = (int32_t)cta_sys.size();
    B->S.cta_sys = a.upload(cta_sys);
    B->S.cta_r0 = a.upload(cta_r0);
    B->S.cta_r1 = a.upload(cta_r1);
    B->S.sys_cta0 = a.upload(sys_cta0);
    if (!B->S.sys_counter) {
        B->S.sys_counter = (unsigned *)a.alloc(sizeof(unsigned) * std::max(1, B->nsys));
        GEMSLR_CUDA(cudaMemset(B->S.sys_counter, 0, sizeof(unsigned) * std::max(1, B->nsys)));
    }
    B->K.partial = (double *)a.alloc(sizeof(double) * std::max(1, B->S.ncta) * (kMaxCols + 1) * kBatchRhs);
}

void ensure_batch_krylov(gemslr_batch_ctx *B, int m) {
    if (m <= B->m_alloc) {             // the buffers of a longer restart serve (strides follow K.m)
        B->K.m = m;
        return;
    }
    if (m + 1 > kMaxCols) fail(GEMSLR_ERR_ARG, "restart length too large");
    Arena &a = B->arena;
    const int64_t L = std::max<int64_t>(1, B->N) * kBatchRhs;
    const int P = std::max(1, B->nsys) * kBatchRhs;
    B->V = (double *)a.alloc(8 * (size_t)L * (m + 1));
    B->Z = (double *)a.alloc(8 * (size_t)L * m);
    if (!B->w) {
        B->w = (double *)a.alloc(8 * L);
        B->x = (double *)a.alloc(8 * L);
        B->b = (double *)a.alloc(8 * L);
        B->r = (double *)a.alloc(8 * L);
        B->vin = (double *)a.alloc(8 * L);
        B->zout = (double *)a.alloc(8 * L);
    }
    BatchKrylov &K = B->K;
    K.npair = P;
    K.m = m;
    K.j = (int32_t *)a.alloc(64);
    K.iters = K.j + 1;
    K.maxit = K.j + 2;
    K.any = K.j + 4;
    auto ai = [&](size_t n) { return (int32_t *)a.alloc(4 * n); };
    auto ad = [&](size_t n) { return (double *)a.alloc(8 * n); };
    K.sys_run = ai(std::max(1, B->nsys));
    K.active = ai(P); K.run = ai(P); K.jdone = ai(P); K.conv = ai(P); K.bad = ai(P); K.its = ai(P); K.restarts = ai(P);
    K.tol = ad(P);
    K.H = ad((size_t)P * (m + 1) * m);
    K.cs = ad((size_t)P * (m + 2)); K.sn = ad((size_t)P * (m + 2)); K.g = ad((size_t)P * (m + 2)); K.y = ad((size_t)P * (m + 2));
    K.hbuf = ad((size_t)P * kMaxCols);
    K.beta = ad(P); K.wn2 = ad(P); K.rn2 = ad(P); K.resid = ad(P);
    GEMSLR_CUDA(cudaMemset(K.H, 0, 8 * (size_t)P * (m + 1) * m));
    B->m_alloc = m;
    if (B->solve_exec) {
        cudaGraphExecDestroy(B->solve_exec);
        B->solve_exec = nullptr;
        cudaGraphDestroy(B->solve_graph);
        B->solve_graph = nullptr;
    }
}

void batch_step(gemslr_batch_ctx *B, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
    const int64_t L = B->N * kBatchRhs;
    batch_apply_layout(B, B->vin, B->zout, st, B->K.sys_run);
    launch_bspmv(B->N, B->A_rp, B->A_ci, B->A_v, B->zout, nullptr, B->w, B->Z, B->K.j, L, st, B->sys_of,
                 B->K.sys_run);
    launch_bgs(1, B->S, B->K, B->V, L, B->w, st);
    launch_bgs(2, B->S, B->K, B->V, L, B->w, st);
    launch_bgs_subnorm(B->S, B->K, B->V, L, B->w, st);
    launch_bgs_final(B->S, B->K, B->V, L, B->w, B->vin, st);
    launch_bstep_end(B->K, h, use_cond, st);
}

void batch_cycle_end(gemslr_batch_ctx *B, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
    const int64_t L = B->N * kBatchRhs;
    launch_blsq(B->K, st);
    launch_bupdate_x(B->S, B->K, B->Z, L, B->x, st);
    launch_bspmv(B->N, B->A_rp, B->A_ci, B->A_v, B->x, B->b, B->r, nullptr, nullptr, 0, st);
    launch_bnorm2(B->S, B->K.partial, B->r, B->K.rn2, st);
    launch_bcycle_end(B->K, h, use_cond, st);
}

// The same kernels in the same order as the solve graph, driven from the
// host (profilers do not see kernels inside conditional graph nodes).
void batch_host_loop(gemslr_batch_ctx *B, cudaStream_t st) {
    const int64_t L = B->N * kBatchRhs;
    auto flag = [&](int i) {
        int32_t v = 0;
        GEMSLR_CUDA(cudaMemcpyAsync(&v, B->K.any + i, 4, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaStreamSynchronize(st));
        return v;
    };
    GEMSLR_CUDA(cudaMemsetAsync(B->x, 0, 8 * L, st));
    GEMSLR_CUDA(cudaMemcpyAsync(B->r, B->b, 8 * L, cudaMemcpyDeviceToDevice, st));
    while (true) {
        launch_bcycle_start(B->K, 0, 0, st);
        launch_bscale(B->S, B->K, B->r, B->V, B->vin, st);
        while (flag(0)) batch_step(B, st, 0, 0);
        batch_cycle_end(B, st, 0, 0);
        if (!flag(1)) break;
    }
}

void ensure_solve_graph_b(gemslr_batch_ctx *B, int m) {
    if (B->solve_exec && B->solve_m == m) return;
    if (B->solve_exec) {                // the kernels of the old graph hold the old restart length
        cudaGraphExecDestroy(B->solve_exec);
        B->solve_exec = nullptr;
        cudaGraphDestroy(B->solve_graph);
        B->solve_graph = nullptr;
    }
    if (!B->cap) GEMSLR_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    cudaStream_t cs = B->cap;
    const int64_t L = B->N * kBatchRhs;
    const uint64_t k0 = launches_total();
    cudaGraph_t g;
    GEMSLR_CUDA(cudaGraphCreate(&g, 0));
    B->solve_graph = g;
    cudaGraphConditionalHandle hc, hs;
    GEMSLR_CUDA(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
    GEMSLR_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    GEMSLR_CUDA(cudaMemsetAsync(B->x, 0, 8 * L, cs));
    GEMSLR_CUDA(cudaMemcpyAsync(B->r, B->b, 8 * L, cudaMemcpyDeviceToDevice, cs));
    cudaGraph_t body_cycle = capture_while_node(cs, hc);
    GEMSLR_CUDA(cudaStreamEndCapture(cs, &g));
    const uint64_t k1 = launches_total();
    GEMSLR_CUDA(cudaGraphConditionalHandleCreate(&hs, body_cycle, 1, cudaGraphCondAssignDefault));
    GEMSLR_CUDA(cudaStreamBeginCaptureToGraph(cs, body_cycle, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_bcycle_start(B->K, hs, 1, cs);
    launch_bscale(B->S, B->K, B->r, B->V, B->vin, cs);
    cudaGraph_t body_step = capture_while_node(cs, hs);
    batch_cycle_end(B, cs, hc, 1);
    GEMSLR_CUDA(cudaStreamEndCapture(cs, &body_cycle));
    const uint64_t k2 = launches_total();
    GEMSLR_CUDA(cudaStreamBeginCaptureToGraph(cs, body_step, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    batch_step(B, cs, hs, 1);
    GEMSLR_CUDA(cudaStreamEndCapture(cs, &body_step));
    const uint64_t k3 = launches_total();
    GEMSLR_CUDA(cudaGraphInstantiate(&B->solve_exec, g, 0));
    B->k_top = k1 - k0;
    B->k_cycle = k2 - k1;
    B->k_step = k3 - k2;
    count_launch(-(int)(k3 - k0));
    B->solve_m = m;
}

void ensure_apply_graph_b(gemslr_batch_ctx *B) {
    if (B->apply_exec) return;
    if (!B->cap) GEMSLR_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    const uint64_t k0 = launches_total();
    GEMSLR_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
    batch_apply_layout(B, B->vin, B->zout, B->cap);
    GEMSLR_CUDA(cudaStreamEndCapture(B->cap, &B->apply_graph));
    GEMSLR_CUDA(cudaGraphInstantiate(&B->apply_exec, B->apply_graph, 0));
    B->k_apply = launches_total() - k0;
    count_launch(-(int)B->k_apply);
}

// Time `fn` on the capture stream (median of 5 after 2 warm-ups), in ms.
double time_ms(cudaStream_t st, const std::function<void()> &fn) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<float> t;
    for (int it = 0; it < 7; ++it) {
        cudaEventRecord(a, st);
        fn();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (it >= 2) t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

namespace gemslr {
// Implemented with the single-system setup (solver.cu): factors + low-rank terms of one system,
// or the host hierarchy of one system with every factor given.
void setup_single_host(const gemslr_csr *A, const gemslr_partition *part, const gemslr_options *opt, Hierarchy &out);
void hierarchy_from_factors(const gemslr_csr *A, const gemslr_partition *part, const gemslr_factors *f,
                            const gemslr_options &opt, Hierarchy &H);
}

namespace {
// Batch set-up: every system's hierarchy from the single-system set-up, or
// (fac non-null, one gemslr_factors per system) from given factors.
gemslr_status setup_batch(int32_t nsys, const gemslr_csr *A, const gemslr_partition *part, const gemslr_factors *fac,
                          const gemslr_options *opt, gemslr_batch *out) {
    if (out) *out = nullptr;
    return bguard([&] {
        if (!out || nsys < 1 || !A || !part) fail(GEMSLR_ERR_ARG, "invalid batch arguments");
        auto t0 = std::chrono::steady_clock::now();
        std::unique_ptr<gemslr_batch_ctx> B(new gemslr_batch_ctx());
        GEMSLR_CUDA(cudaGetDevice(&B->dev));
        if (opt && (opt->dev_alloc == nullptr) != (opt->dev_free == nullptr))
            fail(GEMSLR_ERR_ARG, "dev_alloc and dev_free must be given together");
        if (opt) B->arena.set_allocator(opt->dev_alloc, opt->dev_free, opt->alloc_ctx);
        B->nsys = nsys;
        B->sys.resize(nsys);
        B->base.assign(1, 0);
        gemslr_options o{};
        gemslr_default_options(&o);
        if (opt) o = *opt;
        if (o.shift != 0.0) fail(GEMSLR_ERR_UNSUPPORTED, "the batched path is real (no complex shift)");
        if (fac) {
            for (int s = 0; s < nsys; ++s) hierarchy_from_factors(&A[s], &part[s], &fac[s], o, B->sys[s]);
        } else {
            // the systems' own set-ups (host ILUT, the Arnoldi on the GPU with a host
            // round trip per step) on a few host threads, so that their round trips
            // overlap; the first failure in system order is reported
            int dev = 0;
            GEMSLR_CUDA(cudaGetDevice(&dev));
            std::vector<std::exception_ptr> err(nsys);
            std::atomic<int> next{0};
            std::atomic<bool> failed{false};
            auto work = [&] {
                for (int s; !failed.load() && (s = next.fetch_add(1)) < nsys;) {
                    try {
                        GEMSLR_CUDA(cudaSetDevice(dev));
                        setup_single_host(&A[s], &part[s], opt, B->sys[s]);
                    } catch (...) {
                        err[s] = std::current_exception();
                        failed = true;
                    }
                }
            };
            const int nt = std::min(nsys, 8);
            std::vector<std::thread> pool;
            for (int t = 1; t < nt; ++t) pool.emplace_back(work);
            work();
            for (auto &th : pool) th.join();
            for (auto &e : err)
                if (e) std::rethrow_exception(e);
        }
        for (int s = 0; s < nsys; ++s) {
            if (B->sys[s].cplx) fail(GEMSLR_ERR_UNSUPPORTED, "the batched path is real (complex factors given)");
            if (s > 0 && B->sys[s].nlev != B->sys[0].nlev) fail(GEMSLR_ERR_PARTITION, "all systems need the same nlev");
            B->base.push_back(B->base.back() + B->sys[s].n);
        }
        B->nlev = B->sys[0].nlev;
        B->N = B->base.back();
        Arena &a = B->arena;
        B->err = (int32_t *)a.alloc(16);
        GEMSLR_CUDA(cudaMemset(B->err, 0, 16));
        set_btrsv_smem_limit(dev_smem_optin());
        // batch-wide A (block diagonal), permutation maps
        std::vector<int64_t> rp{0}, perm_g(B->N), nsz(nsys), usr_off(nsys + 1, 0);
        std::vector<int32_t> ci, sys_of(B->N);
        std::vector<double> v;
        int64_t maxd = 1;
        for (int s = 0; s < nsys; ++s) {
            const Hierarchy &h = B->sys[s];
            for (int64_t i = 0; i < h.n; ++i) {
                for (int64_t p = h.Ahat.rp[i]; p < h.Ahat.rp[i + 1]; ++p) {
                    ci.push_back((int32_t)(B->base[s] + h.Ahat.ci[p]));
                    v.push_back(h.Ahat.v[p]);
                }
                rp.push_back((int64_t)ci.size());
                perm_g[B->base[s] + i] = h.perm[i];
                sys_of[B->base[s] + i] = s;
            }
            nsz[s] = h.n;
            for (auto &l : h.lev) maxd = std::max(maxd, l.e - l.s);
            maxd = std::max(maxd, h.n - h.last.s);
        }
        B->A_rp = a.upload(rp);
        B->A_ci = a.upload(ci);
        B->A_v = a.upload(v);
        B->perm_g = a.upload(perm_g);
        B->sys_of = a.upload(sys_of);
        B->nsz = a.upload(nsz);
        B->work = (float *)a.alloc(sizeof(float) * std::max<int64_t>(1, B->N) * kBatchRhs);
        int64_t tot_lev_rows = 1;
        for (int l = 0; l < B->nlev; ++l) {
            int64_t t = 0;
            for (auto &h : B->sys) t += (l + 1 < B->nlev) ? h.lev[l].e - h.lev[l].s : h.n - h.last.s;
            tot_lev_rows = std::max(tot_lev_rows, t);
        }
        B->scratch = (float *)a.alloc(sizeof(float) * tot_lev_rows * kBatchRhs);
        B->lev.resize(B->nlev);
        for (int l = 0; l < B->nlev; ++l) build_batch_level(B.get(), l, l + 1 == B->nlev, B->rows_couple, B->lev[l]);
        build_segments(B.get(), B->rows_krylov);
        ensure_batch_krylov(B.get(), 8);
        // autotuner: rows per CTA of the coupling/low-rank kernels and of the Krylov kernels
        auto tt = std::chrono::steady_clock::now();
        if (!B->cap) GEMSLR_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
        GEMSLR_CUDA(cudaMemsetAsync(B->vin, 0, 8 * B->N * kBatchRhs, B->cap));
        double best = 1e30;
        int best_rows = B->rows_couple;
        for (int rows : {64, 128, 256}) {
            for (int l = 0; l + 1 < B->nlev; ++l) build_batch_level(B.get(), l, false, rows, B->lev[l]);
            const double t = time_ms(B->cap, [&] { batch_apply_layout(B.get(), B->vin, B->zout, B->cap); });
            if (t < best) { best = t; best_rows = rows; }
        }
        B->rows_couple = best_rows;
        for (int l = 0; l + 1 < B->nlev; ++l) build_batch_level(B.get(), l, false, best_rows, B->lev[l]);
        // the Krylov kernels' rows per CTA is not tuned on a proxy: a norm
        // (one column) prefers long CTAs, while the Gram-Schmidt passes over
        // tens of basis columns are bound by load latency and want many CTAs
        // in flight (96 systems x 8 rhs: 2048 rows 173 ms per solve, 1024
        // rows 159 ms, 512 rows 155 ms)
        B->rows_krylov = kKrylovRows;
        build_segments(B.get(), B->rows_krylov);
        GEMSLR_CUDA(cudaStreamSynchronize(B->cap));
        B->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tt).count();
        GEMSLR_CUDA(cudaDeviceSynchronize());
        B->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = B.release();
    });
}
}  // namespace

extern "C" {

gemslr_status gemslr_setup_batch(int32_t nsys, const gemslr_csr *A, const gemslr_partition *part,
                                 const gemslr_options *opt, gemslr_batch *out) {
    return setup_batch(nsys, A, part, nullptr, opt, out);
}

gemslr_status gemslr_setup_batch_from_factors(int32_t nsys, const gemslr_csr *A, const gemslr_partition *part,
                                              const gemslr_factors *f, const gemslr_options *opt,
                                              gemslr_batch *out) {
    if (!f) {
        if (out) *out = nullptr;
        return bguard([&] { fail(GEMSLR_ERR_ARG, "NULL factors"); });
    }
    return setup_batch(nsys, A, part, f, opt, out);
}

static void set_user_layout(gemslr_batch_ctx *B, int nrhs) {
    std::vector<int64_t> off(B->nsys + 1, 0);
    for (int s = 0; s < B->nsys; ++s) off[s + 1] = off[s] + B->sys[s].n * nrhs;
    if (B->usr_off) GEMSLR_CUDA(cudaMemcpy(B->usr_off, off.data(), 8 * off.size(), cudaMemcpyHostToDevice));
    else B->usr_off = B->arena.upload(off);
}

// The batch's device memory belongs to the device it was set up on: a call
// made while another device is current is an argument error, not a fault.
static void require_batch_device(const gemslr_batch_ctx *B) {
    int dev = -1;
    GEMSLR_CUDA(cudaGetDevice(&dev));
    if (dev != B->dev)
        fail(GEMSLR_ERR_ARG, "the batch lives on device " + std::to_string(B->dev) + " but device " +
                                 std::to_string(dev) + " is current");
}

gemslr_status gemslr_batch_apply(gemslr_batch B, const double *r_dev, double *z_dev, int32_t nrhs, void *stream) {
    return bguard([&] {
        if (!B || nrhs < 1 || nrhs > kBatchRhs || !r_dev || !z_dev) fail(GEMSLR_ERR_ARG, "invalid argument");
        require_batch_device(B);
        cudaStream_t st = (cudaStream_t)stream;
        set_user_layout(B, nrhs);
        ensure_apply_graph_b(B);
        launch_bgather(B->N, B->sys_of, B->perm_g, B->usr_off, B->nsz, nrhs, r_dev, B->vin, st);
        GEMSLR_CUDA(cudaGraphLaunch(B->apply_exec, st));
        count_launch((int)B->k_apply);
        launch_bscatter(B->N, B->sys_of, B->perm_g, B->usr_off, B->nsz, nrhs, B->zout, z_dev, st);
        GEMSLR_CUDA(cudaGetLastError());
    });
}

gemslr_status gemslr_batch_fgmres_solve(gemslr_batch B, const double *b_dev, double *x_dev, int32_t nrhs,
                                        const gemslr_solve_opts *opts, gemslr_solve_info *info, void *stream) {
    gemslr_status worst = GEMSLR_OK;
    gemslr_status st_ = bguard([&] {
        if (!B || nrhs < 1 || nrhs > kBatchRhs || !b_dev || !x_dev || !opts || !info)
            fail(GEMSLR_ERR_ARG, "invalid argument");
        if (opts->restart < 1 || opts->maxit < 1 || !(opts->rtol > 0)) fail(GEMSLR_ERR_ARG, "invalid solve options");
        require_batch_device(B);
        auto t0 = std::chrono::steady_clock::now();
        cudaStream_t st = (cudaStream_t)stream;
        const int m = opts->restart;
        ensure_batch_krylov(B, m);
        set_user_layout(B, nrhs);
        // GEMSLR_SOLVE_GRAPH=0 selects the host-driven loop
        const char *env = std::getenv("GEMSLR_SOLVE_GRAPH");
        const bool use_graph = !(env && env[0] == '0');
        if (use_graph) ensure_solve_graph_b(B, m);
        launch_bgather(B->N, B->sys_of, B->perm_g, B->usr_off, B->nsz, nrhs, b_dev, B->b, st);
        launch_bnorm2(B->S, B->K.partial, B->b, B->K.rn2, st);
        launch_binit(B->K, opts->rtol, opts->maxit, st);
        if (use_graph) GEMSLR_CUDA(cudaGraphLaunch(B->solve_exec, st));
        else batch_host_loop(B, st);
        launch_bscatter(B->N, B->sys_of, B->perm_g, B->usr_off, B->nsz, nrhs, B->x, x_dev, st);
        const int P = B->nsys * kBatchRhs;
        std::vector<int32_t> its(P), conv(P), bad(P), rst(P);
        std::vector<double> tol(P), rn2(P);
        int32_t iters = 0, errw = 0;
        GEMSLR_CUDA(cudaMemcpyAsync(its.data(), B->K.its, 4 * P, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(conv.data(), B->K.conv, 4 * P, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(bad.data(), B->K.bad, 4 * P, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(rst.data(), B->K.restarts, 4 * P, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(tol.data(), B->K.tol, 8 * P, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(rn2.data(), B->K.rn2, 8 * P, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(&iters, B->K.iters, 4, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaMemcpyAsync(&errw, B->err, 4, cudaMemcpyDeviceToHost, st));
        GEMSLR_CUDA(cudaStreamSynchronize(st));
        const int ncycle = *std::max_element(rst.begin(), rst.end()) + 1;
        // the host loop's launches counted themselves
        if (use_graph) count_launch((int)(B->k_top + (uint64_t)ncycle * B->k_cycle + (uint64_t)iters * B->k_step));
        if (errw) {
            GEMSLR_CUDA(cudaMemset(B->err, 0, 4));
            fail(GEMSLR_ERR_TIMEOUT, "a bounded wait in the substitution kernel expired");
        }
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        for (int s = 0; s < B->nsys; ++s)
            for (int r = 0; r < nrhs; ++r) {
                const int p = s * kBatchRhs + r;
                gemslr_solve_info &inf = info[s * nrhs + r];
                std::memset(&inf, 0, sizeof(inf));
                inf.iters = its[p];
                inf.restarts = rst[p];
                inf.converged = conv[p];
                const double bn = opts->rtol > 0 ? tol[p] / opts->rtol : 0.0;
                inf.rel_res_true = bn > 0 ? std::sqrt(rn2[p]) / bn : 0.0;
                inf.t_total_ms = ms;
                if (bad[p] && worst == GEMSLR_OK) { worst = GEMSLR_ERR_NAN; g_batch_error = "non-finite values in a solve"; }
                if (!conv[p] && !bad[p] && worst == GEMSLR_OK) {
                    worst = GEMSLR_ERR_NOT_CONVERGED;
                    g_batch_error = "FGMRES reached maxit for at least one system";
                }
            }
    });
    return st_ != GEMSLR_OK ? st_ : worst;
}

gemslr_status gemslr_batch_stats(gemslr_batch B, double *out, int32_t nout) {
    return bguard([&] {
        if (!B || !out || nout < 8) fail(GEMSLR_ERR_ARG, "invalid argument");
        std::fill(out, out + nout, 0.0);
        double nnzf = 0, bytes = 0;
        for (auto &h : B->sys) {
            for (auto &l : h.lev) {
                nnzf += (double)(l.L.nnz() + l.U.nnz());
                bytes += 2.0 * (l.L.nnz() + l.U.nnz()) * (4 + 4) + (l.E.nnz() + l.F.nnz()) * 8.0 +
                         2.0 * (double)(h.n - l.e) * l.k * 2;
            }
            nnzf += (double)(h.last.L.nnz() + h.last.U.nnz());
            bytes += (h.last.L.nnz() + h.last.U.nnz()) * 8.0;
        }
        bytes += (double)B->N * kBatchRhs * 4 * 8;       // vector traffic of the stages, rough
        out[0] = (double)B->nsys;
        out[1] = (double)B->N;
        out[2] = nnzf;
        out[3] = bytes;
        out[4] = B->setup_ms;
        out[5] = B->tune_ms;
        out[6] = B->rows_couple;
        out[7] = B->rows_krylov;
        if (nout > 8) {                    // fewest right-hand sides per substitution CTA (0: global memory)
            int rpc = kBatchRhs;
            for (auto &l : B->lev) rpc = std::min(rpc, l.rpc);
            out[8] = rpc;
        }
        if (nout > 12 && !B->lev.empty()) {   // the first level's sweeps
            const BLevelHost &l0 = B->lev[0];
            out[9] = (double)l0.rows;
            out[10] = (double)l0.l_bytes;
            out[11] = (double)l0.u_bytes;
            out[12] = (double)l0.f_nnz;
        }
    });
}

const char *gemslr_batch_last_error(void) { return g_batch_error.c_str(); }

void gemslr_batch_destroy(gemslr_batch B) { delete B; }

}  // extern "C"
