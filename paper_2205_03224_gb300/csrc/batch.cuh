// Device views of a batch of independent GeMSLR systems solved together with
// kBatchRhs right-hand sides each (the batched workload: many uneven systems,
// one launch per stage of M^{-1} over all of them).
//
// Batch vector layout: the systems one after another, each in its own
// multilevel order; every row holds kBatchRhs consecutive values (one per
// right-hand side): element (row g, rhs r) at g * kBatchRhs + r.
#pragma once

#include "kernels.cuh"

namespace gemslr {

constexpr int kBatchRhs = 8;
constexpr int kBatchWarps = 16;                // consumer warps of the batched substitutions
constexpr int kBatchChunkRows = 4 * kBatchWarps; // 4 rows per warp, 8 lanes (one per rhs) each
constexpr int kBatchTrsvThreads = 32 * (kBatchWarps + 1);
constexpr int kBatchMaxRank = 64;              // k_eff per system in the batched correction
constexpr int kBatchThreads = 256;
constexpr int kKrylovRows = 512;               // batch rows per CTA of the batched Krylov kernels

// One stage level of the batch: the level-l blocks of every system.
struct BatchLevel {
    int32_t nblk;
    const int32_t *order;      // nblk: block of CTA group g (most chunks first)
    const int32_t *blk_sys;    // nblk: system of every block
    // inside a batched solve: nsys flags, 0 when every pair of the system has
    // stopped stepping (its CTAs then return at once); nullptr: apply everything
    const int32_t *live;
    int32_t final_up;          // the first level: its up sweep's result goes to out only
    const int64_t *blk_r0;     // first batch row of every block
    const int32_t *blk_nr;     // rows of every block
    const int64_t *blk_f0;     // first row of the block in the level's F
    ChunkView C;               // L and U chunks of every block (lane-per-row layout)
    const int64_t *F_rp;       // level rows of all systems, in block order
    const int32_t *F_ci;       // batch row
    const float *F_v;
    // tails (one segment per system): E, W, H
    int32_t nseg;
    const int64_t *seg_r0;     // first batch row of the tail of system s
    const int64_t *seg_len;
    const int64_t *seg_e0;     // first row of the segment in the concatenated E
    const int64_t *E_rp;
    const int32_t *E_ci;       // batch row
    const float *E_v;
    const int64_t *seg_w0;     // offset of W_s (seg_len x k_s, column-major)
    const int32_t *seg_k;
    const int64_t *seg_h0;     // offset of H_s (k_s x k_s, column-major)
    const __nv_bfloat16 *W;
    const float *H;
    // work list of the E/W kernels: CTA -> (segment, first tail row); rows per CTA = rows_cta
    int32_t ncta, rows_cta;
    const int32_t *cta_seg;
    const int64_t *cta_i0;
    const int32_t *seg_cta0;   // nseg + 1
    unsigned *seg_counter;     // nseg
    float *partial;            // ncta x kBatchMaxRank x kBatchRhs
    float *u;                  // nseg x kBatchMaxRank x kBatchRhs
    int32_t *err;
};

// Row segments of the batch vector (one per system) for the Krylov kernels.
struct BatchSegs {
    int32_t nsys;
    const int64_t *sys_r0;     // nsys + 1 first batch row of every system
    int32_t ncta;              // work list: CTA -> (system, row range)
    const int32_t *cta_sys;
    const int64_t *cta_r0, *cta_r1;
    const int32_t *sys_cta0;   // nsys + 1
    unsigned *sys_counter;     // nsys
};

// Per (system, rhs) FGMRES state; pair p = s * kBatchRhs + r.
struct BatchKrylov {
    int32_t npair, m;
    int32_t *j;                // current column (all pairs step together)
    int32_t *iters;            // inner steps taken by the batch
    int32_t *any;              // [0] pairs still running in the cycle, [1] pairs still active
    int32_t *maxit;
    int32_t *active;           // pair not yet converged / failed
    int32_t *run;              // pair still stepping in the current cycle
    int32_t *sys_run;          // nsys: some pair of the system still stepping
    int32_t *jdone;            // columns of the pair's current cycle
    int32_t *conv, *bad, *its, *restarts;
    double *tol;               // rtol * ||b_p||
    double *H;                 // npair x (m+1) x m
    double *cs, *sn, *g, *y;   // npair x (m+2)
    double *hbuf;              // npair x kMaxCols
    double *beta;              // npair
    double *wn2;               // npair: ||w||^2 before the first pass
    double *rn2;               // npair: norms of the cycle's starting residual
    double *resid;             // npair: |g_{j+1}|
    double *partial;           // ncta x (kMaxCols + 1) x kBatchRhs
};

}  // namespace gemslr
