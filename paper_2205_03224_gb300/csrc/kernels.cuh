// Device-side views of the GeMSLR hierarchy and the kernel entry points.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace gemslr {

constexpr int kTrsvThreads = 512;
constexpr int kCoupleRows = 256;    // tail rows per CTA in the E / W^T kernel
constexpr int kMaxRank = 160;       // k_eff upper bound in the correction kernels
constexpr int kReduceThreads = 256;
constexpr int kMaxCols = 128;     // Krylov columns per Gram-Schmidt pass (m + 1 <= kMaxCols)

// One triangular factor of one level in the wavefront-sliced layout: the rows
// of a wavefront ("slots") are independent; entry q of slot t of wavefront w
// sits at ent_base[w] + q * (slots in w) + t, so one thread per row reads
// consecutive addresses across a warp.  Columns are block-local.
template <typename VT>
struct TriView {
    const int32_t *blk_wf;     // nblk + 1 : wavefront range of every block
    const int32_t *wf_slot;    // nwf + 1  : slot range of every wavefront
    const int64_t *wf_ent;     // nwf      : first entry of every wavefront
    const int32_t *slot_row;   // block-local row of every slot
    const int32_t *slot_len;   // entries of every slot
    const int32_t *ent_col;    // block-local column
    const VT *ent_val;
};

// Everything one Schur level (or the last level) needs on the device.
template <typename VT, typename WT>
struct LevelView {
    int64_t s, e;              // rows [s, e) of the multilevel order
    int64_t stail;             // n - e
    int32_t nblk;
    const int64_t *blk_row;    // nblk + 1, level-local
    TriView<VT> L, U;          // U without its diagonal
    const VT *dinv;            // 1 / u_ii, level-local
    const int64_t *F_rp;       // d rows
    const int32_t *F_ci;       // global column (>= e)
    const VT *F_v;
    const int64_t *E_rp;       // stail rows
    const int32_t *E_ci;       // level-local column
    const VT *E_v;
    int32_t k;
    const WT *W;               // stail x k, column-major
    const VT *H;               // k x k, column-major
};

// Control block of one FGMRES / Arnoldi step sequence (device memory).
struct KrylovCtl {
    int32_t j;            // current column
    int32_t m;            // restart length
    int32_t stop;         // cycle must end after this step
    int32_t reorth;       // current step needs the second Gram-Schmidt pass
    int32_t breakdown;
    int32_t nonfinite;
    int32_t nreorth;      // count of reorthogonalised steps
    int32_t givens;       // 1: FGMRES (update rotations), 0: Arnoldi
    int32_t force_reorth; // 1: always two passes (Arnoldi)
    int32_t iters;        // total inner iterations
    int32_t maxit;
    int32_t jdone;        // columns of the finished cycle
    double wnorm2;        // ||A z_j||^2 before orthogonalisation
    double beta;          // h_{j+1,j}
    double resid;         // |g_{j+1}|
    double tol_abs;       // rtol * ||b||
    double rnorm2;        // ||r||^2 (restart)
};

}  // namespace gemslr
