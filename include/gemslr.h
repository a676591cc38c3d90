/*
 * gemslr.h -- C ABI of the GB300 GeMSLR-preconditioned FGMRES solve phase.
 *
 * Method: Xu, Kalantzis, Li, Xi, Dillon, Saad, "parGeMSLR: A Parallel
 * Multilevel Schur Complement Low-Rank Preconditioning and Solution Package
 * for General Sparse Matrices" (arXiv 2205.03224).  The problem is A x = b
 * with A large, sparse, possibly non-symmetric (Sec. 1), solved by right-
 * preconditioned restarted FGMRES (Sec. 4.1, Sec. 5) whose preconditioner
 * M^{-1} is the multilevel Schur-complement low-rank (GeMSLR) operator of
 * Alg. 2 built by Alg. 1 over the multilevel vertex-separator reordering of
 * Alg. 3.
 *
 * Conventions for every entry point:
 *  - Host arrays passed in are read during the call only and stay owned by
 *    the caller; the library copies what it keeps.
 *  - Device arrays ("_dev") are caller-owned CUDA device memory on the
 *    current device, FP64, used only on the given stream (NULL = default
 *    stream).  Multi-RHS arrays are column-major with leading dimension n.
 *  - Every call returns a gemslr_status; on failure a thread-local message is
 *    available from gemslr_last_error().  No C++ exception crosses the ABI.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 *  - Levels: nlev counts the Schur levels l = 0..nlev-2 (each with B_l, E_l,
 *    F_l and a rank-k_l correction) plus the last level, the matrix
 *    C_{nlev-2}, which is applied by block-Jacobi incomplete LU of its
 *    diagonal blocks (Sec. 4.3) and has no low-rank term.
 */
#ifndef GEMSLR_H
#define GEMSLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GEMSLR_MAX_LEVELS 16

typedef struct gemslr_ctx *gemslr_handle;   /* opaque, owned by the library */

typedef enum {
    GEMSLR_OK = 0,
    GEMSLR_ERR_ARG = 1,           /* bad argument (NULL, size, option)            */
    GEMSLR_ERR_PARTITION = 2,     /* partition invalid or blocks of B_l coupled    */
    GEMSLR_ERR_ZERO_PIVOT = 3,    /* pivot clamped while options.strict_pivots set */
    GEMSLR_ERR_NOT_CONVERGED = 4, /* FGMRES hit maxit (the paper's "F")           */
    GEMSLR_ERR_NAN = 5,           /* NaN/Inf in b or during the iteration          */
    GEMSLR_ERR_TIMEOUT = 6,       /* a bounded device wait expired                 */
    GEMSLR_ERR_CUDA = 7,          /* CUDA runtime error                            */
    GEMSLR_ERR_NOMEM = 8,         /* host or device allocation failed              */
    GEMSLR_ERR_UNSUPPORTED = 9    /* valid request the library does not implement  */
} gemslr_status;

/* Host CSR matrix, 0-based, columns ascending within a row. */
typedef struct {
    int64_t n;                /* rows = columns                                   */
    const int64_t *rowptr;    /* n + 1                                            */
    const int32_t *colind;    /* rowptr[n]                                        */
    const double *val;        /* rowptr[n]                                        */
} gemslr_csr;

/*
 * Multilevel partition (Alg. 3): perm lists the original index of every
 * unknown in the multilevel order (new -> old).  Level l owns the contiguous
 * range [level_ptr[l], level_ptr[l+1]); its blocks are given by
 * block_ptr[o_l .. o_l + nblk[l]] relative to level_ptr[l], where
 * o_l = sum_{i<l} (nblk[i] + 1).  For Schur levels the blocks must be
 * uncoupled in |A| + |A^T| (the vertex-separator property, Sec. 3); the
 * last level's blocks are the block-Jacobi blocks (Sec. 4.3).
 */
typedef struct {
    int32_t nlev;
    const int32_t *perm;       /* n                        */
    const int64_t *level_ptr;  /* nlev + 1                 */
    const int32_t *nblk;       /* nlev                     */
    const int64_t *block_ptr;  /* sum(nblk) + nlev         */
} gemslr_partition;

/* Precision of the preconditioner application (FGMRES is FP64 in both). */
enum { GEMSLR_PREC_FP64 = 0, GEMSLR_PREC_MIXED = 1 };
/* Incomplete factorisation of the diagonal blocks: ILU(0) or ILUT on the host
 * (blocks on a pool of host threads), ILU(0) on the GPU (level-scheduled,
 * one CTA per block; factors bit-identical to GEMSLR_ILU0; every row of A
 * needs its diagonal entry, else ARG), or ILUT on the GPU (one warp per
 * block, the block's rows in order since the fill depends on the values;
 * factors bit-identical to GEMSLR_ILUT; needs 0 <= ilut_lfil <= 64, else
 * ARG). */
enum { GEMSLR_ILU0 = 0, GEMSLR_ILUT = 1, GEMSLR_ILU0_DEVICE = 2, GEMSLR_ILUT_DEVICE = 3 };

typedef struct {
    int32_t ilu_kind;             /* GEMSLR_ILU0, _ILUT, _ILU0_DEVICE, _ILUT_DEVICE */
    double ilut_tau;              /* ILUT drop tolerance (relative to ||a_i||_2)    */
    int32_t ilut_lfil;            /* ILUT fill per row in L and in U (<0: no cap)   */
    int32_t rank[GEMSLR_MAX_LEVELS]; /* k_l per Schur level (0 = no correction)     */
    int32_t precision;            /* GEMSLR_PREC_FP64 or GEMSLR_PREC_MIXED          */
    double arnoldi_tol;           /* Ritz accuracy for the low-rank term (1e-2)     */
    int32_t arnoldi_max_cycles;   /* thick-restart cycles (20)                      */
    int32_t strict_pivots;        /* nonzero: a clamped pivot fails the setup      */
    /* Device allocator for everything a handle keeps on the GPU (factors,
     * Krylov workspace, graphs' buffers): dev_alloc(bytes, alloc_ctx) returns a
     * device pointer aligned to at least 256 bytes, or NULL on failure (the call
     * then fails with NOMEM); dev_free(ptr, alloc_ctx) releases it when the
     * handle is destroyed, after the device has finished all the handle's
     * work.  Both NULL (the default): cudaMalloc / cudaFree.
     * Setting only one of them is an ARG error.  The callbacks run on the
     * calling thread, inside the library's calls. */
    void *(*dev_alloc)(size_t bytes, void *alloc_ctx);
    void (*dev_free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    /* Set-up of the low-rank corrections: GEMSLR_LOWRANK_ARNOLDI (thick-restart
     * Krylov-Schur, Sec. 4.2; the default) or GEMSLR_LOWRANK_RANDOMIZED (the
     * block / randomized variant that Sec. 6 names as future work: subspace
     * iteration on a seeded random s x 2k block with lowrank_power passes,
     * then Rayleigh-Ritz with the same selection of the wanted values). */
    int32_t lowrank_method;
    int32_t lowrank_power;        /* subspace-iteration passes (randomized; 1)   */
    /* Complex diagonal shift of the incomplete factorisations (Sec. 5.2.3, the
     * paper's Helmholtz experiments use 0.05): with shift != 0 every diagonal
     * block of every B_l and of the last level is factored as B + i alpha I,
     * alpha = shift * sum_i |a_ii| / n (E, F and C are not shifted), the
     * corrections come from the Arnoldi in complex arithmetic (W H W^H, complex
     * Schur form), and the handle is complex: gemslr_zapply and
     * gemslr_zfgmres_solve apply and solve in complex FP64; the real entry
     * points refuse it (ARG).  A complex handle needs precision FP64, a host
     * ilu_kind (ILU0 or ILUT) and the Arnoldi set-up, else UNSUPPORTED.  0: the
     * real method (the default). */
    double shift;
} gemslr_options;
enum { GEMSLR_LOWRANK_ARNOLDI = 0, GEMSLR_LOWRANK_RANDOMIZED = 1 };

/* Fill *opt with the defaults: ILUT(1e-3, 10), rank 0, FP64, 1e-2, 20 cycles,
 * Arnoldi set-up of the corrections (1 pass when randomized is chosen), no
 * complex shift. */
void gemslr_default_options(gemslr_options *opt);

/*
 * Geometric multilevel partition (Alg. 3 with a p-way vertex separator from
 * recursive coordinate bisection; the last level ordered by reverse
 * Cuthill-McKee and cut into p_last chunks, Sec. 4.3).  coords: n x 3 int32
 * grid coordinates, row-major.  p must be a power of two.  Output arrays are
 * caller-allocated: perm (n), level_ptr (nlev+1), nblk (nlev),
 * block_ptr ((nlev-1)*(p+1) + p_last + 1).
 */
gemslr_status gemslr_partition_geometric(const gemslr_csr *A, const int32_t *coords,
                                         int32_t nlev, int32_t p, int32_t p_last,
                                         int32_t *perm, int64_t *level_ptr, int32_t *nblk,
                                         int64_t *block_ptr);

/*
 * Local order inside the diagonal blocks (Sec. 3.2: each B_l may be permuted
 * locally, the multilevel structure unchanged).  For every block of the
 * levels first_level .. nlev-1 (the last level included), the block's entries
 * of part->perm are sorted stably by the colour key 8 t + c of their vertex,
 * t = (floor(x/2) mod 2) + 2 (floor(y/2) mod 2) + 4 (floor(z/2) mod 2) the
 * colour of its 2 x 2 x 2 tile and c = (x mod 2) + 2 (y mod 2) + 4 (z mod 2)
 * its point colour (coords: n x 3 int32 grid coordinates, row-major).  Each
 * class is an independent set of a 5- or 7-point stencil, so the blocks'
 * triangular factors get fewer, wider wavefronts.  perm_out (n, caller-owned)
 * receives the new permutation and may be part->perm itself; level_ptr, nblk
 * and block_ptr stay valid.  Errors: ARG (NULL, first_level outside
 * 0..nlev), PARTITION (inconsistent offsets).
 */
gemslr_status gemslr_local_order(int64_t n, const int32_t *coords, const gemslr_partition *part,
                                 int32_t first_level, int32_t *perm_out);

/*
 * Setup (Alg. 1): permute A, factor every diagonal block of every B_l and of
 * the last level, then bottom-up (Sec. 4.2) compute the rank-k_l correction
 * W_l [(I - R_l)^{-1} - I] W_l^T from thick-restart Arnoldi on
 * G_l = E_l (U_l^{-1} L_l^{-1}) F_l C_l^{-1} (Sec. 2.3), with C_l^{-1} the
 * GPU application of the levels below.  Uses the current CUDA device.
 * Errors: ARG, PARTITION (blocks coupled), ZERO_PIVOT (strict_pivots),
 * CUDA, NOMEM.  On success *out owns all device memory it uses.
 */
gemslr_status gemslr_setup(const gemslr_csr *A, const gemslr_partition *part,
                           const gemslr_options *opt, gemslr_handle *out);

/* One CSR piece of the hierarchy in the multilevel order (host, 0-based). */
typedef struct {
    int64_t nrows, ncols;
    const int64_t *rowptr;
    const int32_t *colind;
    const double *val;
} gemslr_mat;

/*
 * Factors of one Schur level l, in level-local numbering:
 *  L: d_l x d_l strictly lower (unit diagonal implied), block diagonal;
 *  U: d_l x d_l upper including its diagonal, block diagonal;
 *  E: s_l x d_l (rows: the tail [level_ptr[l+1], n) minus level_ptr[l+1]);
 *  F: d_l x s_l;
 *  W: s_l x k column-major, H = (I - R_k)^{-1} - I: k x k column-major.
 */
typedef struct {
    gemslr_mat L, U, E, F;
    int32_t k;
    const double *W;
    const double *H;
    /* Complex factors (the complex shift, Sec. 5.2.3): imaginary parts of
     * L.val, U.val (nnz each), W (s x k) and H (k x k), same layouts; NULL: 0.
     * Factors with any imaginary part make a complex handle. */
    const double *L_im, *U_im, *W_im, *H_im;
} gemslr_level_factors;

typedef struct {
    int32_t nlev;
    const gemslr_level_factors *levels;   /* nlev - 1 Schur levels              */
    gemslr_mat last_L, last_U;            /* last level, block diagonal         */
    const double *last_L_im, *last_U_im;  /* imaginary parts (NULL: 0)          */
} gemslr_factors;

/*
 * Build a handle from factors computed elsewhere (checkpoint/resume, or a
 * reference computation): nothing is factored, the permuted A is still
 * formed for the FGMRES products.  Factors with imaginary parts give a
 * complex handle (FP64 only).  Same errors as gemslr_setup.
 */
gemslr_status gemslr_setup_from_factors(const gemslr_csr *A, const gemslr_partition *part,
                                        const gemslr_factors *f, const gemslr_options *opt,
                                        gemslr_handle *out);

/*
 * Sizes of the handle's factors (for gemslr_export_factors buffers; a complex
 * handle exports its imaginary parts into the *_im buffers, which must then
 * all be given, and cannot be saved to a factor file: UNSUPPORTED):
 * counts[0] = nlev; then per Schur level l, 9 entries starting at 1 + 9*l:
 * nnz(L), nnz(U), nnz(E), nnz(F), k, d_l, s_l, level_ptr[l], level_ptr[l+1];
 * then nnz(last_L), nnz(last_U), size of the last level.  ncounts must be at
 * least 4 + 9*(nlev-1).
 */
gemslr_status gemslr_factor_sizes(gemslr_handle h, int64_t *counts, int64_t ncounts);

/*
 * Copy the factors out (host).  The caller fills the pointer fields of every
 * gemslr_mat / W / H in *f with buffers of the sizes reported by
 * gemslr_factor_sizes (rowptr nrows+1, colind/val nnz, W s*k, H k*k); the
 * library writes into them.
 */
gemslr_status gemslr_export_factors(gemslr_handle h, gemslr_factors *f);

/*
 * Factor files (checkpoint / resume of the set-up, Alg. 1): gemslr_save_factors
 * writes every factor of the handle (per Schur level L, U, E, F, k, W, H; the
 * last level's L and U) to `path` in a little-endian binary layout;
 * gemslr_load_factors reads such a file and builds a handle like
 * gemslr_setup_from_factors for the same A and partition (nothing is
 * factored).  Errors: ARG (NULL argument, the file cannot be opened, written
 * or read, is not a factor file, is corrupt, or belongs to another matrix size
 * or partition), plus those of gemslr_setup_from_factors.
 */
gemslr_status gemslr_save_factors(gemslr_handle h, const char *path);
gemslr_status gemslr_load_factors(const gemslr_csr *A, const gemslr_partition *part, const char *path,
                                  const gemslr_options *opt, gemslr_handle *out);

/*
 * z = M^{-1} r (Alg. 2) for nrhs right-hand sides in the ORIGINAL ordering:
 * z = P M_hat^{-1} P^T r.  r_dev, z_dev: n x nrhs column-major device arrays
 * (may not alias).  Asynchronous on `stream`.  The device that was current
 * when the handle was set up must be current (this applies to
 * gemslr_apply_static and gemslr_fgmres_solve too); otherwise ARG.
 */
gemslr_status gemslr_apply(gemslr_handle h, const double *r_dev, double *z_dev, int32_t nrhs,
                           void *stream);

/*
 * Inner GMRES at the root level (Alg. 2 step 9).  With steps > 0, every
 * application of M^{-1} (gemslr_apply, gemslr_apply_static and the FGMRES
 * solves) replaces the root level's y2 = M_S^{-1} z2 by `steps` steps of
 * right-preconditioned GMRES from y2 = 0 on S_hat_0 y2 = z2, where
 * S_hat_0 = C_0 - E_0 U_0^{-1} L_0^{-1} F_0 is the inexact Schur complement of
 * the root level (Sec. 2.4) and M_S^{-1} its preconditioner: the level-0
 * low-rank correction (eq. gemslr6) followed by the levels below.  The Arnoldi
 * vectors use the application's precision with FP64 sums; a happy breakdown
 * (h_{j+1,j} <= 1e-14 ||S_hat_0 z_j||) ends the steps early.  M^{-1} becomes
 * nonlinear; FGMRES (flexible) then uses classical Gram-Schmidt with a second
 * pass.  steps = 0 restores the standard application.  The first call with
 * steps > 0 allocates the Arnoldi storage (about (2 steps + 3) x (n - level_ptr[1])
 * vector entries plus a copy of the rows [level_ptr[1], n) of P^T A P).
 * Errors: ARG (steps outside [0, 8], no Schur level, or the learned stage
 * enabled: the two are exclusive), CUDA, NOMEM.
 */
gemslr_status gemslr_set_inner_steps(gemslr_handle h, int32_t steps);

typedef struct {
    int32_t restart;     /* FGMRES cycle length m                               */
    int32_t maxit;       /* total inner iterations (1,000 in the paper)         */
    double rtol;         /* stop when ||b - A x|| <= rtol ||b|| (true residual) */
    int32_t ortho;       /* single system only: 0 = automatic (delayed
                            reorthogonalisation, one reduction per step, where
                            M^{-1} is linear, i.e. without the learned stage);
                            1 = classical Gram-Schmidt with a second pass when
                            the first cancels (three reductions per step)     */
} gemslr_solve_opts;

typedef struct {
    int32_t iters;            /* inner iterations taken                         */
    int32_t restarts;         /* completed cycles that did not converge        */
    int32_t converged;        /* 1 if the true residual met rtol                */
    int32_t reorth;           /* iterations that needed a second orthogonalisation */
    double rel_res_est;       /* |g_{j+1}| / ||b|| at exit                      */
    double rel_res_true;      /* ||b - A x|| / ||b|| at exit                    */
    double t_total_ms;        /* wall time of the solve call                    */
} gemslr_solve_info;

/*
 * Solve A x = b by restarted right-preconditioned FGMRES(m) with x_0 = 0 and
 * M^{-1} from the handle.  b_dev, x_dev: n x nrhs column-major device arrays in
 * the original ordering; info: nrhs entries (host).  Synchronises `stream`.
 * With delayed reorthogonalisation the handle also runs work on a second,
 * internal stream of its own (created on first use), forked from and joined
 * back into `stream` within every step, so that the next direction's
 * reorthogonalisation overlaps the application of M^{-1}; the call returns
 * with both idle.  Calls on one handle must not overlap.  The whole solve is
 * one CUDA graph with conditional nodes; with the environment variable
 * GEMSLR_SOLVE_GRAPH=0 the same kernels run in the same order from a host
 * loop instead (for profilers, which do not see kernels inside conditional
 * nodes; the iterates are identical).
 * Returns NOT_CONVERGED (with info filled) when maxit is reached, NAN when b
 * or the iteration is not finite.
 */
gemslr_status gemslr_fgmres_solve(gemslr_handle h, const double *b_dev, double *x_dev,
                                  int32_t nrhs, const gemslr_solve_opts *opts,
                                  gemslr_solve_info *info, void *stream);

/*
 * Complex application and solve (handles set up with a complex shift, or from
 * complex factors; Sec. 5.2.3): the same operations as gemslr_apply and
 * gemslr_fgmres_solve in complex FP64.  Vectors are n x nrhs column-major
 * arrays of complex values stored as (re, im) double pairs (the C99
 * double _Complex layout), in the original ordering.  gemslr_zapply:
 * z = M^{-1} r, asynchronous on `stream`, r and z may not alias.
 * gemslr_zfgmres_solve: restarted right-preconditioned FGMRES(m) (Sec. 4.1)
 * with x_0 = 0, inner products v^H w, classical Gram-Schmidt with a second
 * pass, complex Givens rotations; stops on the true residual
 * ||b - A x|| <= rtol ||b||.  opts->ortho is ignored.  Synchronises `stream`.
 * Errors: ARG (a real handle, NULL or invalid arguments, another device
 * current), NOT_CONVERGED (info filled), NAN, CUDA, TIMEOUT.
 */
gemslr_status gemslr_zapply(gemslr_handle h, const double *r_dev, double *z_dev, int32_t nrhs, void *stream);
gemslr_status gemslr_zfgmres_solve(gemslr_handle h, const double *b_dev, double *x_dev, int32_t nrhs,
                                   const gemslr_solve_opts *opts, gemslr_solve_info *info, void *stream);

/*
 * Statistics: out[0..] = n, nlev, nclamped pivots, nnz(A), nnz of all
 * factors, algorithmic bytes per M^{-1} application, setup ms, device bytes,
 * then per level: d_l, s_l, k_l, nnz(L_l)+nnz(U_l), L wavefronts, U wavefronts.
 * nout: capacity of out (8 + 6*nlev suffices).
 */
gemslr_status gemslr_get_stats(gemslr_handle h, double *out, int32_t nout);

/* Message of the last failed call on this thread ("" if none). */
const char *gemslr_last_error(void);

/* Free the handle and its device memory (NULL is accepted). */
void gemslr_destroy(gemslr_handle h);

/*
 * Batched solve phase: many independent systems (each with its own CSR,
 * multilevel partition and setup, Alg. 1) handled together with up to
 * GEMSLR_BATCH_RHS right-hand sides each.  Every stage of M^{-1} (Alg. 2) is
 * one launch over all systems; FGMRES runs for every (system, rhs) pair in
 * lock step, the whole solve being one CUDA graph (GEMSLR_SOLVE_GRAPH=0: a
 * host loop, as for gemslr_fgmres_solve); a system whose pairs have all
 * stopped is skipped by the rest of the cycle's steps.  The preconditioner is
 * applied in FP32 (W in BF16, FP32 accumulation); Krylov vectors, the
 * least-squares problems and residuals are FP64.  All systems need the same
 * nlev; ranks up to 64.
 *
 * Vector layout of r/z/b/x: the systems one after another, system s a
 * column-major n_s x nrhs block in its original ordering.
 * gemslr_setup_batch: A and part are arrays of nsys entries; opt applies to all.
 * gemslr_batch_apply: z = M_s^{-1} r for every system and rhs (captured graph).
 * gemslr_batch_fgmres_solve: info has nsys * nrhs entries (system-major).
 * Both return ARG when a device other than the one the batch was set up on
 * is current.
 * gemslr_batch_stats: out[0..7] = nsys, total rows, factor nonzeros, bytes of one
 * application (approximate), setup ms, autotuning ms, rows per CTA of the
 * coupling kernels (tuned) and of the Krylov kernels (512); with nout > 8, out[8] = the fewest
 * right-hand sides a substitution CTA handles (8, 4, 2 or 1: a level whose
 * largest block's vector for 8 right-hand sides does not fit in shared memory
 * splits them over several CTAs; 0: a block too large even for 1 keeps its
 * vector in global memory); with nout > 12, out[9..12] = the first level's
 * block rows (all systems), bytes of its stored L chunks and of its U chunks,
 * and the nonzeros of its F (what one down and one up sweep of that level
 * must read).
 */
#define GEMSLR_BATCH_RHS 8
typedef struct gemslr_batch_ctx *gemslr_batch;
gemslr_status gemslr_setup_batch(int32_t nsys, const gemslr_csr *A, const gemslr_partition *part,
                                 const gemslr_options *opt, gemslr_batch *out);
/*
 * Batch from factors computed elsewhere (Alg. 1 done by another program, or
 * a checkpoint): f is an array of nsys gemslr_factors, one per system, in the
 * layout of gemslr_setup_from_factors; nothing is factored and no Arnoldi
 * runs, only the autotuner.  The factors are copied (caller-owned).  Errors:
 * ARG (NULL f, a level count, shape or rank that does not match the system's
 * partition, a rank above 64), plus those of gemslr_setup_batch.
 */
gemslr_status gemslr_setup_batch_from_factors(int32_t nsys, const gemslr_csr *A, const gemslr_partition *part,
                                              const gemslr_factors *f, const gemslr_options *opt,
                                              gemslr_batch *out);
gemslr_status gemslr_batch_apply(gemslr_batch b, const double *r_dev, double *z_dev, int32_t nrhs,
                                 void *stream);
gemslr_status gemslr_batch_fgmres_solve(gemslr_batch b, const double *b_dev, double *x_dev, int32_t nrhs,
                                        const gemslr_solve_opts *opts, gemslr_solve_info *info,
                                        void *stream);
gemslr_status gemslr_batch_stats(gemslr_batch b, double *out, int32_t nout);
const char *gemslr_batch_last_error(void);
void gemslr_batch_destroy(gemslr_batch b);

/*
 * Allocation-free M^{-1} (the paper has no counterpart; an interface
 * addition).  Same result as gemslr_apply with nrhs = 1, for callers that
 * cannot allocate device memory when they apply the preconditioner: code
 * running while a stream is captured into a CUDA graph (cudaMalloc is not
 * allowed during a global-mode capture), callers whose own pool or allocator
 * owns all device memory, and latency-critical loops that must not enter the
 * allocator.  gemslr_apply may allocate its permutation buffers on its first
 * call; this entry point never calls cudaMalloc, cudaFree or any allocating
 * routine: the permuted copies of r and z live in a fixed device array of
 * 2 x 2,097,152 doubles (32 MiB) that every GPU loading the library holds
 * until the process exits.  Limit: n <= 2,097,152, larger handles are
 * rejected with GEMSLR_ERR_ARG.  The first call on a device looks up the
 * array's device address (with that device current), so make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents; every call overwrites all n entries it reads, so
 * nothing needs clearing, but calls that overlap on the GPU (different
 * streams, or different handles at once) race on it.  Instrumentation
 * (gemslr_profile_enable) must be off.
 */
gemslr_status gemslr_apply_static(gemslr_handle h, const double *r_dev, double *z_dev, void *stream);

/*
 * Learned interface correction (an addition; the paper has no counterpart).
 * At the deepest Schur level l* = nlev-2, after M^{-1}'s recursion has
 * produced y2 from z2, the stage computes rho = z2 - S_hat y2 with
 * S_hat = C - E (U^{-1} L^{-1}) F of that level (Sec. 2.4) and adds
 * (||rho||/d) * net(rho/||rho||), net a 4-layer 27-tap 3-D convolution network
 * over the level's unknowns (BF16 weights, FP32 accumulation), d the mean
 * |diagonal| of S_hat.  The application becomes nonlinear, which flexible
 * GMRES tolerates (Sec. 5 set-up).
 * gemslr_learned_train: coords (n x 3 grid coordinates, original order) give
 * the sites; generates npairs (rho, S_hat^{-1} rho) pairs with rho = z - S_hat
 * M_S^{-1} z (z ~ U[-1,1) from splitmix64(seed ^ 0x5eed), M_S^{-1} the
 * method's own level-l* application), trains with Adam on the relative
 * squared error, enables the stage; loss_history (epochs entries, may be
 * NULL) receives the mean training loss per epoch.
 * gemslr_learned_enable: switch the stage on or off.
 * gemslr_learned_info: out[0..3] = sites, channels, d, parameter count.
 * gemslr_learned_params: get (get != 0) or set the FP32 master parameters,
 * flattened as W_0, b_0, ..., W_3, b_3 with W_l[t][c_in][c_out] (t = 27 taps,
 * t = (dz+1)*9 + (dy+1)*3 + (dx+1)); setting refreshes the BF16 copies.
 * gemslr_learned_loss_grad: mean loss and parameter gradients (same layout)
 * for nb given scaled inputs x and targets y (nb x sites, row-major).
 */
typedef struct {
    int32_t channels;   /* hidden channels (<= 32)          */
    int32_t npairs;     /* training pairs                   */
    int32_t epochs;
    int32_t batch;
    double lr;          /* Adam step size                   */
    uint64_t seed;
} gemslr_learned_opts;
gemslr_status gemslr_learned_train(gemslr_handle h, const int32_t *coords, const gemslr_learned_opts *o,
                                   double *loss_history);
gemslr_status gemslr_learned_enable(gemslr_handle h, int32_t on);
gemslr_status gemslr_learned_info(gemslr_handle h, double *out);
gemslr_status gemslr_learned_params(gemslr_handle h, int32_t get, double *params, int64_t n);
gemslr_status gemslr_learned_loss_grad(gemslr_handle h, int32_t nb, const double *x, const double *y, double *loss,
                                       double *grad);

/*
 * Instrumentation (not part of the method; process-wide, thread-safe).
 * gemslr_kernel_launches: number of CUDA kernels this library has launched.
 * gemslr_profile_enable: with on != 0 every instrumented launch is bracketed
 * by CUDA events on its stream (adds host overhead; for measurement runs).
 * gemslr_profile_read: synchronises the recorded events and returns the
 * number of kernel names; writes up to maxn totals (ms) and launch counts,
 * and the names, newline-separated, into names[len].
 * gemslr_profile_reset: drops the accumulated totals.
 */
uint64_t gemslr_kernel_launches(void);
/*
 * gemslr_selftest_wait (no counterpart in the paper): exercises the bounded
 * device waits every staged kernel relies on.  One CTA waits on an mbarrier
 * that nothing completes, once with the suspending wait and once with the
 * polling wait, each bounded by `cycles` SM clock cycles (> 0).  Returns
 * GEMSLR_ERR_TIMEOUT when both waits gave up and the context is still usable
 * afterwards (the expected outcome), GEMSLR_ERR_CUDA on a CUDA error,
 * GEMSLR_ERR_ARG if a wait returned or cycles <= 0.  Uses the default stream
 * and synchronises the device.
 */
gemslr_status gemslr_selftest_wait(int64_t cycles);
void gemslr_profile_enable(int32_t on);
void gemslr_profile_reset(void);
int32_t gemslr_profile_read(char *names, size_t len, double *ms, int64_t *counts, int32_t maxn);

#ifdef __cplusplus
}
#endif
#endif /* GEMSLR_H */
