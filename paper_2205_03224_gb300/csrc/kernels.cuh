// Device-side views of the GeMSLR hierarchy and the kernel entry points.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "zcomplex.cuh"

namespace gemslr {

constexpr int kTrsvThreads = 512;
constexpr int kCoupleRows = 256;    // tail rows per CTA in the E / W^T kernel
constexpr int kMaxRank = 160;       // k_eff upper bound in the correction kernels
constexpr int kReduceThreads = 256;
constexpr int kMaxCols = 160;     // Krylov columns per Gram-Schmidt pass (m + 1 <= kMaxCols)

// Triangular factors of one level as a sequence of "chunks" per block: the L
// chunks of a block in wavefront (level-set) order, then its U chunks.  A
// chunk holds <= kChunkRows independent rows of one wavefront and is one
// contiguous, 16-byte aligned byte range of <= StageBytesOf<VT> bytes:
//   int32 {nrows, S, upper, more}     S = entry slots per row; more = 1 when
//                                     another slice of the same layout follows
//                                     in the same chunk (FP32: up to kMaxSlices
//                                     consecutive wavefront slices per chunk
//                                     when they fit)
//   int32 rows[pad4(nrows)]           block-local row of every slot
//   int32 lens[pad4(nrows)]           entries of every slot
//   int32 cols[pad4(S*nrows)]         block-local columns
//   VT    vals[S*nrows] padded to 16 bytes: -t_ij in L chunks, -u_ij/u_ii in
//         U chunks (formed in FP64, rounded once), so that a row is
//         x_i = x_i * d_i + sum_j vals_ij x_j with d_i = 1 (L) or 1/u_ii (U)
//   VT    dinv[nrows]  padded to 16 bytes (U chunks: 1/u_ii)
// Entry q of row slot t sits at
//   FP32 (one lane per row, S = maxlen):          q*nrows + t
//   FP64 (four lanes per row, S = 4*ceil(maxlen/4)): ((q/4)*nrows + t)*4 + q%4
// so a warp always reads consecutive addresses.  The chunks of a block move
// into a shared-memory ring of kRingData bytes CPG at a time: group g (chunks
// CPG*g onwards, contiguous in global memory) is one bulk copy into ring slot
// g % (kRingData / (CPG*StageBytesOf<VT>)), and a chunk is found in its slot by
// skipping the chunks before it (their sizes follow from their headers).
// The FP32 substitutions move kGroupChunks chunks per copy (one per consumer
// warp); the FP64 and batched ones, whose warps share every chunk, move one.
constexpr int kStageBytes = 4096;
constexpr int kGroupChunks = 4;
constexpr int kRingData = 16 * kStageBytes;
constexpr int kMaxSlots = kRingData / kStageBytes;
constexpr int kConsumerWarps = 4;
constexpr int kChunkRows = 32;
constexpr int kTrsvThreads2 = 32 * (kConsumerWarps + 1);
constexpr int kRingBytes = kRingData + 2 * kMaxSlots * 8 + 64;   // ring + mbarriers + flags
template <typename VT> struct LanesPerRow { static constexpr int value = 4; };
template <> struct LanesPerRow<float> { static constexpr int value = 1; };
// Largest chunk of a value type: complex chunks (16-byte values) are twice as
// large, so that a typical wavefront still fits in one chunk (one hand-off).
template <typename VT> struct StageBytesOf { static constexpr int value = kStageBytes; };
template <> struct StageBytesOf<zc> { static constexpr int value = 2 * kStageBytes; };
// FP32 chunks (single system) hold up to kMaxSlices consecutive wavefront
// slices in 8 KB, so that a consumer warp hands the sweep on once per four
// wavefronts (a hand-off costs more than a slice solved by the same warp).
template <> struct StageBytesOf<float> { static constexpr int value = 2 * kStageBytes; };
constexpr int kMaxSlices = 4;

struct ChunkView {
    const unsigned char *data;
    const int64_t *off;        // nchunk + 1 byte offsets into data
    const int32_t *blk_chunk;  // nblk + 1 chunk range of every block
};

// Everything one Schur level (or the last level) needs on the device.
template <typename VT, typename WT>
struct LevelView {
    int64_t s, e;              // rows [s, e) of the multilevel order
    int64_t stail;             // n - e
    int32_t nblk;
    int32_t max_slots;         // longest chunk row (entry slots) of the level's factors
    const int64_t *blk_row;    // nblk + 1, level-local
    ChunkView C;               // L and U of every block (see above)
    int32_t *err;              // device error word (1: a bounded wait expired)
    const int64_t *F_rp;       // d rows
    const int32_t *F_ci;       // global column (>= e)
    const VT *F_v;
    const int32_t *F_rows;     // level-local rows with F entries, ascending (so grouped by block)
    const int32_t *F_blk;      // nblk + 1 ranges of every block's rows in F_rows
    const int64_t *E_rp;       // stail rows
    const int32_t *E_ci;       // level-local column
    const VT *E_v;
    int32_t k;
    const WT *W;               // stail x k, column-major
    const VT *H;               // k x k, column-major
};

// The low-rank term W u of the previous level (Alg. 2 step 7: the right-hand
// side of level l+1 is z2 + W u), applied by the kernels that first read each
// row of that level's tail instead of by a separate pass: row g of the
// multilevel order takes sum_c W[g - row0 + c*ld] u[c].  W == nullptr: none.
template <typename VT, typename WT>
struct PendingLowRank {
    const WT *W = nullptr;
    const VT *u = nullptr;
    int64_t ld = 0, row0 = 0;
    int32_t k = 0;
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
    int32_t restarts;     // completed cycles that did not converge
    int32_t converged;    // true residual met tol_abs
    double rnorm;         // ||b - A x|| after the last cycle
    double nu;            // delayed CGS2: norm of the reorthogonalised direction of this step
    double btil;          // delayed CGS2: lagged norm of the next direction
    double btil_prev;     // delayed CGS2: btil of the step before (row j of column j-1)
    double gam_pre;       // delayed CGS2: vt.vt of the current direction (formed beside M^{-1})
};

// Device buffers of FGMRES with delayed reorthogonalisation (one reduction
// per step): the unrotated Hessenberg matrix, the rotated one with its
// rotations and right-hand side, the triangular R relating the stored
// directions' preconditioned vectors to those of the final basis, and the
// per-step coefficient vectors.
struct DgsBufs {
    double *Hraw;          // (m+1) x m, column-major
    double *Hrot;          // (m+1) x m, column-major (least-squares factor)
    double *cs, *sn, *g;   // rotations and rotated right-hand side
    double *R;             // (m+1) x (m+1), column-major, upper triangular
    double *a;             // kMaxCols: V^T (direction) of this step
    double *apre;          // kMaxCols: the same, formed beside M^{-1} (k_dgs_fix_adots)
    double *coef;          // kMaxCols: projection coefficients of the next direction
    double *hprev;         // kMaxCols: first-pass column of the previous step
};

// Inner GMRES at the root level (Alg. 2 step 9): up to kMaxInner steps of
// right-preconditioned GMRES on S_hat_0 y2 = z2, S_hat_0 = C_0 - E_0 U^-1 L^-1 F_0
// (Sec. 2.4), preconditioned by the level-0 correction and the levels below.
constexpr int kMaxInner = 8;

struct InnerCtl {
    int32_t steps;         // Arnoldi steps taken (columns of H in use)
    int32_t done;          // 1: z2 = 0 or a happy breakdown ended the steps
    double beta;           // ||z2||
    double wn0;            // ||S_hat z_j|| before orthogonalisation (breakdown test)
    double h2[kMaxInner + 1];  // second-pass coefficients of the current step
    double c[kMaxInner];   // least-squares coefficients of y2 = sum_j c_j z_j
};

// Device state of the inner GMRES.  Vectors have the tail length m = n - e0
// (rows [e0, n) of the multilevel order).
template <typename VT>
struct InnerView {
    int64_t m;                 // n - e0
    int64_t e0;                // first tail row
    int32_t k;                 // steps per application (<= kMaxInner)
    const int64_t *rp;         // rows [e0, n) of A_hat: m + 1 offsets
    const int32_t *ci;         // global columns
    const VT *v;
    VT *V;                     // m x (k + 1), column-major: Arnoldi basis
    VT *Z;                     // m x k: preconditioned basis (M_S^-1 v_j)
    VT *w;                     // m
    double *H;                 // (kMaxInner + 1) x kMaxInner, column-major
    double *partial;           // grid x (kMaxInner + 2), column-major
    unsigned *counter;
    InnerCtl *ctl;
    int grid;                  // CTAs of the reduction kernels
};

}  // namespace gemslr
