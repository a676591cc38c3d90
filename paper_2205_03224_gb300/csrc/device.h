// Device-side state of a GeMSLR handle and the launch wrappers of kernels.cu.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "learned.cuh"

namespace gemslr {

void cuda_check(cudaError_t e, const char *what);
#define GEMSLR_CUDA(x) ::gemslr::cuda_check((x), #x)

// ---- instrumentation -------------------------------------------------------------
// Every launch wrapper counts its launch; with profiling on, ProfScope
// brackets a launch with CUDA events on its stream and the elapsed time is
// accumulated per kernel name when the profile is read.
void count_launch(int n = 1);
struct ProfScope {
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
    int slot;
    cudaStream_t st;
};

void profile_enable(bool on);
bool profile_enabled();
void profile_reset();
int profile_read(char *names, size_t len, double *ms, int64_t *counts, int maxn);
uint64_t launches_total();

// ---- launchers (kernels.cu) --------------------------------------------------
// pl: the previous level's pending W u (MODE 0 only; default: none).
template <typename VT, typename WT>
void launch_trsv(const LevelView<VT, WT> &lv, int mode, int smem_rows, const IoT<VT> *in, VT *work,
                 IoT<VT> *out_final, VT *scratch, cudaStream_t st,
                 const PendingLowRank<VT, WT> &pl = PendingLowRank<VT, WT>());
template <typename VT, typename WT> void set_trsv_smem_limit(int bytes);
template <typename VT, typename WT>
void launch_couple(const LevelView<VT, WT> &lv, const IoT<VT> *in, VT *work, VT *partial, unsigned *counter,
                   VT *u, cudaStream_t st, const PendingLowRank<VT, WT> &pl = PendingLowRank<VT, WT>());
void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t st);
void launch_scatter(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t st);
void launch_zero(int64_t n, double *x, cudaStream_t st);
void launch_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x,
                 const double *b, double *y, int lanes, cudaStream_t st, double *zcol = nullptr,
                 const KrylovCtl *ctl = nullptr);
void launch_gs_dots(int64_t len, const double *V, int64_t ldv, const double *w, double *partial, unsigned *counter,
                    KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *hbuf, int grid,
                    cudaStream_t st);
// w = A z (z also stored in column j of zcol), then the first Gram-Schmidt pass
// (rows split over `grid` CTAs; for matrices with short rows).
void launch_gs_spmv_dots(int64_t len, const int64_t *rp, const int32_t *ci, const double *av, const double *z,
                         double *zcol, const double *V, int64_t ldv, double *w, double *partial, unsigned *counter,
                         KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *hbuf, int grid,
                         cudaStream_t st);
void launch_gs_sub(int64_t len, double *V, int64_t ldv, double *w, double *partial, unsigned *counter,
                   KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *h2buf, int grid,
                   cudaStream_t st, double *vcopy = nullptr);
void launch_gs_sub2(int64_t len, double *V, int64_t ldv, double *w, const double *h2, double *partial,
                    unsigned *counter, KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, int grid,
                    cudaStream_t st);
void launch_gs_scale(int64_t len, double *V, int64_t ldv, const double *w, const KrylovCtl *ctl, double *vcopy,
                     cudaStream_t st);
void launch_gs_next(KrylovCtl *ctl, cudaStream_t st);
// FGMRES with delayed reorthogonalisation (see kernels.cu): step reduction,
// step update, cycle close, and the two back substitutions (R may be null).
void launch_dgs_dots(int64_t len, const int64_t *rp, const int32_t *ci, const double *av, const double *z, double *zcol,
                     const double *V, int64_t ldv, const double *vt, double *w, double *partial, unsigned *counter,
                     KrylovCtl *ctl, const DgsBufs &B, int grid, cudaStream_t st);
void launch_dgs_next(int64_t len, double *V, int64_t ldv, double *vt, const double *w, const KrylovCtl *ctl,
                     const DgsBufs &B, cudaStream_t st);
// reorthogonalisation of step ctl->j + off (nothing when negative), `grid` CTAs;
// exclusive: CTAs that never share an SM with a substitution CTA
void launch_dgs_fix(int64_t len, double *V, int64_t ldv, const KrylovCtl *ctl, const DgsBufs &B, int off, int grid,
                    bool exclusive, cudaStream_t st);
// the previous step's reorthogonalisation and V^T vt, vt . vt of the current
// direction (partials: `grid` x (kMaxCols + 2)), beside M^{-1}
void launch_dgs_fix_adots(int64_t len, double *V, int64_t ldv, const double *vt, double *partial, unsigned *counter,
                          KrylovCtl *ctl, const DgsBufs &B, int grid, cudaStream_t st);
// the Hessenberg column, rotations and stopping test of the step (one CTA)
void launch_dgs_tail(KrylovCtl *ctl, const DgsBufs &B, cudaStream_t st);
// kernel attributes of the Krylov kernels (call before any capture)
void prepare_krylov_kernels();
void launch_dgs_close(int64_t len, const double *V, int64_t ldv, const double *vt, double *partial, unsigned *counter,
                      KrylovCtl *ctl, const DgsBufs &B, int grid, cudaStream_t st);
void launch_lsq2(const KrylovCtl *ctl, const double *H, const double *g, const double *R, double *y, cudaStream_t st);
// Two bounded waits on an mbarrier nothing completes (see gemslr_selftest_wait).
void launch_wait_selftest(long long limit, int32_t *gave_up, cudaStream_t st);
void launch_norm2(int64_t len, const double *x, double *partial, unsigned *counter, double *out, int grid,
                  cudaStream_t st);
void launch_scale_by_norm(int64_t len, const double *x, const double *n2, double *v, cudaStream_t st,
                          double *vcopy = nullptr);
void launch_cycle_start(KrylovCtl *ctl, double *g, const double *n2, cudaStream_t st);
void launch_lsq(const KrylovCtl *ctl, const double *H, const double *g, double *y, cudaStream_t st);
void launch_update_x(int64_t len, const double *Z, int64_t ldz, const KrylovCtl *ctl, const double *y, double *x,
                     cudaStream_t st);
void launch_cycle_start_g(KrylovCtl *ctl, double *g, const double *n2, cudaGraphConditionalHandle h, cudaStream_t st);
void launch_step_end_g(KrylovCtl *ctl, cudaGraphConditionalHandle h, cudaStream_t st);
void launch_cycle_end_g(KrylovCtl *ctl, const double *n2r, cudaGraphConditionalHandle h, cudaStream_t st);
void launch_basis_rotate(int64_t len, const double *V, int64_t ldv, int mm, const double *Q, int kk, double *out,
                         cudaStream_t st);
// B = V^T Z (b x b, column-major) for s x b column-major V, Z (lowrank_rand.cu).
void launch_gram(int64_t s, int b, const double *V, const double *Z, double *B, cudaStream_t st);

// ---- host-side conversions and the chunk layout of the substitutions ---------------
template <typename T> inline T cast_to(double v);
template <> inline double cast_to<double>(double v) { return v; }
template <> inline float cast_to<float>(double v) { return (float)v; }
template <> inline __nv_bfloat16 cast_to<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
template <> inline zc cast_to<zc>(double v) { return zc(v); }
template <typename T> inline std::vector<T> convert(const std::vector<double> &x) {
    std::vector<T> y(x.size());
    for (size_t i = 0; i < x.size(); ++i) y[i] = cast_to<T>(x[i]);
    return y;
}

template <typename VT>
struct ChunkHost {
    std::vector<unsigned char> data;
    std::vector<int64_t> off{0};
    std::vector<int32_t> blk_chunk{0};
    int maxwf_L = 0, maxwf_U = 0;
    int max_slots = 0;                 // largest S of any slice
};

// Chunks (layout in kernels.cuh) of the block-diagonal factors L, U of one
// level: slices of at most max_rows row slots, up to max_slices (1 ..
// kMaxSlices) consecutive slices per chunk of at most stage_bytes.
template <typename VT>
void build_chunks(const Csr &L, const Csr &U, const std::vector<int64_t> &bp, ChunkHost<VT> &out, int max_rows,
                  int max_slices, int stage_bytes);

// ---- device memory arena ------------------------------------------------------------
class Arena {
  public:
    ~Arena();
    // caller's device allocator (both null: cudaMalloc / cudaFree); before any alloc
    void set_allocator(void *(*a)(size_t, void *), void (*f)(void *, void *), void *ctx) {
        alloc_fn_ = a;
        free_fn_ = f;
        ctx_ = ctx;
    }
    void *alloc(size_t bytes);
    template <typename T> T *upload(const std::vector<T> &v) {
        T *p = (T *)alloc(v.size() * sizeof(T));
        if (!v.empty()) GEMSLR_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return p;
    }
    size_t bytes() const { return total_; }

  private:
    std::vector<void *> ptrs_;
    size_t total_ = 0;
    void *(*alloc_fn_)(size_t, void *) = nullptr;
    void (*free_fn_)(void *, void *) = nullptr;
    void *ctx_ = nullptr;
};

// One level in device memory (value type VT, low-rank storage WT).
template <typename VT, typename WT>
struct DevLevel {
    LevelView<VT, WT> view{};
    int smem_rows = 0;          // dynamic shared memory rows of the trsv kernel (0 = global)
    int nwf_L = 0, nwf_U = 0;   // wavefront counts (max over blocks)
    int64_t nnz_tri = 0;
    int64_t nchunks = 0;
};

// Inner GMRES of the root level (inner.cu); k = 0: the standard application.
template <typename VT>
struct DevInner {
    int k = 0;
    InnerView<VT> iv{};
    VT *work2 = nullptr;          // n: Arnoldi operands in the multilevel order
    int64_t *zero_rp = nullptr;   // m + 1 zeros: an empty E_0 (u = H_0 W_0^T v only)
};

template <typename VT>
void launch_inner_norm(const InnerView<VT> &iv, const VT *z2, cudaStream_t st);
template <typename VT>
void launch_inner_start(const InnerView<VT> &iv, const VT *z2, VT *work2, cudaStream_t st);
template <typename VT>
void launch_inner_spmv_dots(const InnerView<VT> &iv, int j, const VT *work2, cudaStream_t st);
template <typename VT>
void launch_inner_sub_dots(const InnerView<VT> &iv, int j, cudaStream_t st);
template <typename VT>
void launch_inner_scale(const InnerView<VT> &iv, int j, VT *work2, cudaStream_t st);
template <typename VT>
void launch_inner_lsq(const InnerView<VT> &iv, cudaStream_t st);
template <typename VT>
void launch_inner_combine(const InnerView<VT> &iv, VT *work, double *out_final, cudaStream_t st);

template <typename VT, typename WT>
struct DevHierarchy {
    std::vector<DevLevel<VT, WT>> lev;   // Schur levels
    DevLevel<VT, WT> last;
    VT *work = nullptr;                  // n, M^{-1} work vector (mixed precision)
    VT *scratch = nullptr;               // max d_l, trsv up-sweep without shared memory
    VT *partial = nullptr;               // couple-kernel partial sums
    unsigned *counter = nullptr;
    VT *u = nullptr;                     // kMaxRank
    int32_t *err = nullptr;              // device error word of the substitution kernels
    LearnedStage<VT> *learned = nullptr; // optional learned correction at the deepest Schur level
    DevInner<VT> inner;                  // optional inner GMRES at the root level (Alg. 2 step 9)
};

// Learned-stage glue (learned.cu).
template <typename VT> void learned_save(const LearnedStage<VT> &L, int64_t e, const VT *work, cudaStream_t st);
template <typename VT> void learned_rho_and_update(const LearnedStage<VT> &L, int64_t e, VT *work, cudaStream_t st);
template <typename VT> void launch_cast_out(int64_t n, const VT *src, double *dst, cudaStream_t st);
void net_forward(NetDev &net, int N, const float *x0, float *const zs[4], float *const hs[3], cudaStream_t st);
void net_backward(NetDev &net, int N, const float *x0, float *const zs[4], float *const hs[3], float *dout,
                  float *gbuf0, float *gbuf1, float *part, int nchunk, cudaStream_t st);
void net_adam(NetDev &net, float lr, cudaStream_t st);
void net_sync_bf16(NetDev &net, cudaStream_t st);
// Shared-memory limits of the tensor-core convolutions (once per device, before any capture).
void net_kernels_init();
void launch_uniform(uint64_t seed, int64_t count, double *out, cudaStream_t st);
void launch_dgemm(int M, int N, int K, const double *A, const double *B, double *C, cudaStream_t st);
void launch_scale_pairs(int S, int count, const double *R, const double *T, double d, float *X, float *Y,
                        cudaStream_t st);
void launch_loss(int S, int N, const float *out, const float *tgt, float *dout, float *loss, cudaStream_t st);

// ---- complex-shifted hierarchy (complex.cu, Sec. 5.2.3) -----------------------------
// Device copy of a complex host hierarchy with its Krylov workspace; the
// low-rank terms are built on the device (bottom-up) when compute_lowrank.
struct ZState;
ZState *z_create(Hierarchy &h, Arena &a, const gemslr_options &opt, const int64_t *A_rp, const int32_t *A_ci,
                 const double *A_v, const int32_t *perm, int smem_limit, int sms, bool compute_lowrank);
void z_destroy(ZState *z);
void z_wavefronts(const ZState *z, int l, int &wl, int &wu);   // l = nlev - 1: the last level
// z = M^{-1} r, complex vectors in the original ordering (nrhs columns of n)
void z_apply(ZState *z, const zc *r, zc *out, int32_t nrhs, cudaStream_t st);
// complex FGMRES for one right-hand side; msg receives the reason of a non-OK status
gemslr_status z_solve(ZState *z, const zc *b, zc *x, const gemslr_solve_opts &o, gemslr_solve_info &inf,
                      std::string &msg, cudaStream_t st);

// Build the device copy of a host hierarchy.
template <typename VT, typename WT>
void upload_hierarchy(const Hierarchy &h, Arena &arena, DevHierarchy<VT, WT> &d, int smem_limit_bytes);

// Attach the low-rank term of a host level to its device level.
template <typename VT, typename WT>
void set_lowrank(DevLevel<VT, WT> &d, const HostLevel &hl, Arena &a);

// Apply levels >= from (Alg. 2 recursion entered at level `from`).  With
// `in` non-null the right-hand side is read from it (FP64, multilevel
// order); otherwise from the tail of `work` starting at level `from`.
// out_final (optional) receives the FP64 result of every level.  pend0: a
// W u term to add to the right-hand side of level `from` (from > 0).  With
// from == 0 and inner steps set, the root level runs Alg. 2 step 9.
template <typename VT, typename WT>
void apply_levels(DevHierarchy<VT, WT> &d, int from, const IoT<VT> *in, VT *work, IoT<VT> *out_final,
                  cudaStream_t st, const PendingLowRank<VT, WT> &pend0 = PendingLowRank<VT, WT>());

// Allocate (once) and switch on the inner GMRES with k steps (k = 0: off).
template <typename VT, typename WT>
void setup_inner(const Hierarchy &h, Arena &a, DevHierarchy<VT, WT> &d, int k, int sms);

// z = M^{-1} r in the multilevel order.  `in` FP64 (length n), `out` FP64.
// start_level > 0 applies the sub-hierarchy of levels >= start_level to the
// tail held in d.work (used by the Arnoldi operator), with in/out ignored.
template <typename VT, typename WT>
void apply_hierarchy(DevHierarchy<VT, WT> &d, int64_t n, const double *in, double *out, cudaStream_t st);

}  // namespace gemslr
