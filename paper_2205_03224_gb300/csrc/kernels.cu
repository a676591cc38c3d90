// CUDA kernels of the GeMSLR solve phase for sm_103a.
//
// Preconditioner application (Alg. 2), per Schur level l:
//   k_trsv   (down)  z1 = U^-1 L^-1 b1          one CTA per diagonal block of B_l,
//                    level-scheduled substitutions on a shared-memory copy of
//                    the block's vector (Sec. 4.2: the p block solves are
//                    independent);
//   k_couple         z2 = b2 - E_l z1 and the partial sums of W_l^T z2; the last
//                    CTA to finish reduces them in a fixed order and forms
//                    u = H_l (W_l^T z2), H_l = (I - R_l)^-1 - I (eq. gemslr5);
//   W_l u            (the right-hand side u2 + z2 of level l+1) is added by the
//                    kernels that first read each tail row: the next level's
//                    down sweep and coupling kernel, or the last level;
//   last level       k_trsv on the block-Jacobi blocks (Sec. 4.3);
//   k_trsv   (up)    y1 = z1 - U^-1 L^-1 (F_l y2), F_l y2 formed row by row as
//                    the right-hand side of the forward sweep.
// FGMRES (Sec. 4.1): CSR SpMV; for a linear M^-1 delayed classical
// Gram-Schmidt with reorthogonalisation (k_dgs_*: one reduction after each
// product, the second pass and the previous basis vector beside M^-1), else
// classical Gram-Schmidt with a second pass when the first one cancels
// (Daniel-Gragg-Kaufman-Stewart test, k_gs_*); Givens update of the Hessenberg
// least-squares problem, solution update.  Reductions are per-CTA partial sums
// finished by the last CTA in a fixed order, so results are deterministic run
// to run.
#include <cstdio>

#include "device.h"
#include "ptx.cuh"

namespace gemslr {

namespace {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename VT, typename WT> __device__ __forceinline__ VT wval(WT w) { return (VT)to_f(w); }
template <> __device__ __forceinline__ double wval<double, double>(double w) { return w; }
template <> __device__ __forceinline__ zc wval<zc, zc>(zc w) { return w; }
// an entry of W^H (the correction is W H W^H; for real data W^T)
template <typename VT, typename WT> __device__ __forceinline__ VT wval_h(WT w) { return wval<VT, WT>(w); }
template <> __device__ __forceinline__ zc wval_h<zc, zc>(zc w) { return conj(w); }

// Row g's share of the previous level's W u (see PendingLowRank): sixteen
// columns at a time with all their loads issued first (columns past k load
// the last column again and are multiplied by zero).  u is read through L2:
// the coupling kernel that reads it also rewrites it in its finisher.
template <typename VT, typename WT>
__device__ __forceinline__ VT pending_row(const PendingLowRank<VT, WT> &pl, int64_t g) {
    const WT *w = pl.W + (g - pl.row0);
    VT a0 = 0, a1 = 0;
    for (int c0 = 0; c0 < pl.k; c0 += 16) {
        WT wv[16];
        VT uv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int c = min(c0 + q, pl.k - 1);
            wv[q] = w[(int64_t)c * pl.ld];
            uv[q] = c0 + q < pl.k ? ldcg(pl.u + c) : (VT)0;
        }
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
            a0 += wval<VT, WT>(wv[q]) * uv[q];
            a1 += wval<VT, WT>(wv[q + 1]) * uv[q + 1];
        }
    }
    return a0 + a1;
}


// ---- level-scheduled substitutions over one block --------------------------
// One CTA per diagonal block.  Warp kConsumerWarps is the producer: it
// streams the block's chunks (see kernels.cuh) into a shared-memory ring,
// CPG chunks per bulk copy completing on an mbarrier.  The
// consumer warps keep the block's vector x in shared memory (or global memory
// for blocks that do not fit) and, chunk by chunk, compute
//   x_i = (x_i - sum_j T_ij x_j) * (U ? 1/u_ii : 1)
// with the rows of a chunk spread over the consumer warps, lane per row.
// MODE 0: right-hand side from `in` (FP64 user vector) or `work`; result in work.
// MODE 1: right-hand side F y2 (gathered from work's tail); work[rows] -= result.
template <typename VT, typename WT, int MODE, bool SMEM, int NE>
__global__ void __launch_bounds__(kTrsvThreads2)
k_trsv(const LevelView<VT, WT> lv, const IoT<VT> *__restrict__ in, VT *__restrict__ work,
       IoT<VT> *__restrict__ out_final, VT *__restrict__ scratch, const PendingLowRank<VT, WT> pl) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *ring = smem;
    // FP32: kGroupChunks chunks per copy, one per consumer warp; FP64: one
    constexpr int CPG = LanesPerRow<VT>::value == 1 ? kGroupChunks : 1;
    constexpr int SB = StageBytesOf<VT>::value;
    constexpr int kSlots = kRingData / (CPG * SB);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kRingData);
    uint64_t *empty = full + kSlots;
    uint64_t *cbar = empty + kSlots;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(cbar + 1);
    VT *xs_smem = reinterpret_cast<VT *>(smem + kRingBytes);

    const int b = blockIdx.x;
    const int64_t r0 = lv.blk_row[b];
    const int nr = (int)(lv.blk_row[b + 1] - r0);
    if (nr == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = lv.C.blk_chunk[b], c1 = lv.C.blk_chunk[b + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&full[s], 1);
            // FP32 chunks are released by one consumer warp, FP64 chunks by all of them
            mbar_init(&empty[s], CPG * (LanesPerRow<VT>::value == 1 ? 1 : kConsumerWarps));
        }
        mbar_init(cbar, kConsumerWarps);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumerWarps) {            // producer warp
        produce_chunks<CPG, SB>(lv.C.data, lv.C.off, c0, c1, ring, full, empty, abort_flag, lv.err, lane);
        return;
    }

    // consumer warps: every chunk ends with the same named barrier, so a warp
    // whose wait expired keeps the barrier count of the others (no deadlock)
    const int ct = threadIdx.x;                        // 0 .. 32*kConsumerWarps-1
    constexpr int NC = 32 * kConsumerWarps;
    VT *mine = work + lv.s + r0;
    VT *xs = SMEM ? xs_smem : (MODE == 1 ? scratch + r0 : mine);
    if (MODE == 1) {
        // right-hand side F y2: zero, then the (few) block rows with F entries,
        // one thread per row so that their index and value loads overlap
        for (int i = ct; i < nr; i += NC) xs[i] = (VT)0;
        consumer_barrier();
        // four rows per thread at a time, each step's loads for all of them in
        // flight together (row ids, row extents, the first two entries, x)
        const int f1 = lv.F_blk[b + 1];
        for (int t0 = lv.F_blk[b] + ct; t0 < f1; t0 += 4 * NC) {
            int64_t g[4], pa[4], pb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) g[u] = t0 + u * NC < f1 ? lv.F_rows[t0 + u * NC] : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                pa[u] = g[u] >= 0 ? lv.F_rp[g[u]] : 0;
                pb[u] = g[u] >= 0 ? lv.F_rp[g[u] + 1] : 0;
            }
            int32_t cc[4][2];
            VT vv[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const bool live = pa[u] + q < pb[u];
                    const int64_t pq = live ? pa[u] + q : pa[u];
                    cc[u][q] = g[u] >= 0 ? lv.F_ci[pq] : 0;
                    vv[u][q] = live ? lv.F_v[pq] : (VT)0;
                }
            VT xv[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < 2; ++q) xv[u][q] = g[u] >= 0 ? work[cc[u][q]] : (VT)0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (g[u] < 0) continue;
                VT acc = vv[u][0] * xv[u][0] + vv[u][1] * xv[u][1];
                for (int64_t p = pa[u] + 2; p < pb[u]; ++p) acc += lv.F_v[p] * work[lv.F_ci[p]];
                xs[g[u] - r0] = acc;
            }
        }
    } else if (pl.W) {
        // right-hand side z2 + W u of the previous level (MODE 0, never the first level)
        for (int i = ct; i < nr; i += NC) xs[i] = mine[i] + pending_row<VT, WT>(pl, lv.s + r0 + i);
    } else if (in || SMEM) {
        // eight independent loads in flight per thread
        const IoT<VT> *src_d = in ? in + lv.s + r0 : nullptr;
        for (int i0 = ct; i0 < nr; i0 += 8 * NC) {
            VT v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * NC;
                v[u] = i < nr ? (src_d ? (VT)src_d[i] : mine[i]) : (VT)0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u * NC < nr) xs[i0 + u * NC] = v[u];
        }
    }
    consumer_barrier();
    if constexpr (LanesPerRow<VT>::value == 1) {
        // FP32: the consumer warps take the chunks in turn, one lane per row,
        // each loading its next chunk into registers while the others work.
        consume_chunks_round_robin<VT, NE, SB>(ring, full, empty, abort_flag, c1 - c0, xs, warp, lane);
    } else {
        bool aborted = false;
        const int r = lane >> 2, sub = lane & 3;
        const unsigned char *base = nullptr;
        for (int c = c0; c < c1; ++c) {
            const int k = c - c0;
            base = aborted ? nullptr : next_chunk<VT, CPG, SB>(ring, full, abort_flag, k, base);
            if (!aborted && !base) {
                aborted = true;
                *abort_flag = 1;
            }
            if (!aborted) {
                const int *hdr = reinterpret_cast<const int *>(base);
                const int nrow = hdr[0], S = hdr[1], upper = hdr[2];
                const int pr = (nrow + 3) & ~3;
                const int *rows = hdr + 4;
                const int *lens = rows + pr;
                const int *cols = lens + pr;
                const VT *vals = reinterpret_cast<const VT *>(cols + (size_t)S * nrow);
                const int per = (nrow + kConsumerWarps - 1) / kConsumerWarps;   // rows of this warp (<= 8)
                if (warp * per < nrow) {                                       // idle warps skip the FP64 work
                    // x_row = x_row d + sum_j v_j x_j with v_j = -t_row,j (d = 1, L) or
                    // -u_row,j / u_row,row (d = 1 / u_row,row, U): the padded slots hold
                    // column 0 and value 0, so every lane loads its first four entries
                    // unconditionally, all loads before the arithmetic, and adds them in
                    // two short chains (dependent FP64 operations are slow on this part);
                    // inactive lanes read row slot 0 and their sums are discarded
                    const int t = warp * per + r;
                    const bool active = r < per && t < nrow;
                    const int tt = active ? t : 0;
                    const int kq = S >> 2;
                    const int row = rows[tt];
                    int cq[4];
                    VT vq[4], xq[4];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {                            // slots past S: column 0, value 0
                        const int e = (kk * nrow + tt) * 4 + sub;
                        cq[kk] = kk < kq ? cols[e] : 0;
                        vq[kk] = kk < kq ? vals[e] : (VT)0;
                    }
                    VT a0 = 0;
                    if (sub == 0) {
                        a0 = xs[row];
                        if (upper) a0 *= vals[(size_t)S * nrow + tt];          // dinv follows vals
                    }
                    VT a1 = 0;
                    if constexpr (IsComplex<VT>::value) {
                        // a complex product is four FP64 FMAs: skip the slots past kq
                        // (uniform over the chunk)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) xq[kk] = kk < kq ? xs[cq[kk]] : (VT)0;
                        if (kq > 0) a0 += vq[0] * xq[0];
                        if (kq > 1) a1 = vq[1] * xq[1];
                        if (kq > 2) a0 += vq[2] * xq[2];
                        if (kq > 3) a1 += vq[3] * xq[3];
                    } else {
                        // FP64: all four slots, no branches (padded slots add 0 * x_0)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) xq[kk] = xs[cq[kk]];
                        a1 = vq[1] * xq[1];
                        a0 += vq[0] * xq[0];
                        a1 += vq[3] * xq[3];
                        a0 += vq[2] * xq[2];
                    }
                    for (int kk = 4; kk < kq; ++kk) {                          // rows of more than 16 entries
                        const int e = (kk * nrow + tt) * 4 + sub;
                        a0 += vals[e] * xs[cols[e]];
                    }
                    VT acc = a0 + a1;
                    acc += shfl_xor(acc, 1);
                    acc += shfl_xor(acc, 2);
                    if (active && sub == 0) xs[row] = acc;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[chunk_slot<CPG, SB>(k)]);
            }
            consumer_barrier();
        }
    }
    consumer_barrier();
    if (*abort_flag) {
        if (ct == 0) atomicExch(lv.err, 1);
        return;
    }
    for (int i = ct; i < nr; i += NC) {
        VT y = xs[i];
        if (MODE == 1) y = mine[i] - y;
        if (SMEM || MODE == 1) mine[i] = y;
        if (out_final) out_final[lv.s + r0 + i] = (IoT<VT>)y;
    }
}

// z2 = b2 - E z1 on rows [row0, row1) of the tail, then partial W^T z2 (W^H z2
// for the complex hierarchy).
template <typename VT, typename WT>
__global__ void __launch_bounds__(kCoupleRows)
k_couple(const LevelView<VT, WT> lv, const IoT<VT> *__restrict__ in, VT *__restrict__ work,
         VT *__restrict__ partial, unsigned *__restrict__ counter, VT *u_out,
         const PendingLowRank<VT, WT> pl) {
    __shared__ VT zs[kCoupleRows];
    __shared__ VT ts[kMaxRank];
    __shared__ int last;
    const int64_t i0 = (int64_t)blockIdx.x * kCoupleRows;
    const int64_t i1 = min(i0 + (int64_t)kCoupleRows, lv.stail);
    const int64_t i = i0 + threadIdx.x;
    VT z = 0;
    if (i < i1) {
        z = in ? (VT)in[lv.e + i] : work[lv.e + i];
        if (pl.W) z += pending_row<VT, WT>(pl, lv.e + i);
        // the row's first two E entries with all their loads together, then the rest
        const int64_t pa = lv.E_rp[i], pb = lv.E_rp[i + 1];
        int32_t cc[2];
        VT vv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const bool live = pa + q < pb;
            const int64_t pq = live ? pa + q : pa;
            cc[q] = pb > pa ? lv.E_ci[pq] : 0;
            vv[q] = live ? lv.E_v[pq] : (VT)0;
        }
        const VT x0 = work[lv.s + cc[0]], x1 = work[lv.s + cc[1]];
        z -= vv[0] * x0;
        z -= vv[1] * x1;
        for (int64_t p = pa + 2; p < pb; ++p) z -= lv.E_v[p] * work[lv.s + lv.E_ci[p]];
        work[lv.e + i] = z;
    }
    zs[threadIdx.x] = z;
    const int k = lv.k;
    if (k == 0) return;
    __syncthreads();
    // partial W^T z2: warp w takes columns w, w+nw, w+2nw, w+3nw together, each
    // lane its eight rows of every one of them, all 32 loads before any FMA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t nr = i1 - i0;
    static_assert(kCoupleRows == 256, "eight rows per lane");
    for (int cb = warp; cb < k; cb += 4 * nwarp) {
        WT wv[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = min(cb + u * nwarp, k - 1);
            const WT *wc = lv.W + (int64_t)c * lv.stail + i0;
#pragma unroll
            for (int q = 0; q < 8; ++q) wv[u][q] = wc[min((int64_t)(lane + 32 * q), nr - 1)];
        }
        VT acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc[u] = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[u] += wval_h<VT, WT>(wv[u][q]) * zs[lane + 32 * q];   // zs = 0 past i1
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = cb + u * nwarp;        // uniform over the warp
            if (c < k) {
                const VT t = warp_sum(acc[u]);
                if (lane == 0) partial[(int64_t)c * gridDim.x + blockIdx.x] = t;
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // u = H t: every thread's row of H is loaded while the partials are reduced
    constexpr int kHPre = sizeof(VT) == 4 ? 32 : 16;
    VT hrow[kHPre];
    const int c = threadIdx.x;
#pragma unroll
    for (int d = 0; d < kHPre; ++d) hrow[d] = (c < k && d < k) ? lv.H[c + (int64_t)d * k] : (VT)0;
    reduce_columns<VT>(partial, (int)gridDim.x, k, ts);
    for (int cc2 = c; cc2 < k; cc2 += blockDim.x) {
        VT acc = 0;
        if (cc2 == c) {
#pragma unroll
            for (int d = 0; d < kHPre; ++d) acc += hrow[d] * (d < k ? ts[d] : (VT)0);
            for (int d = kHPre; d < k; ++d) acc += lv.H[cc2 + (int64_t)d * k] * ts[d];
        } else {
            for (int d = 0; d < k; ++d) acc += lv.H[cc2 + (int64_t)d * k] * ts[d];
        }
        u_out[cc2] = acc;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// ---- bounded-wait self-test ---------------------------------------------------
// An mbarrier that nothing ever completes: warp 0 waits on it with the
// suspending wait, warp 1 with the polling wait, both bounded by `limit`
// clock cycles.  gave_up[w] = 1 when warp w's wait expired (it must).
__global__ void k_wait_selftest(long long limit, int32_t *gave_up) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const bool got = warp == 0 ? wait_bounded(&bar, 0, &abort_flag, limit)
                               : poll_bounded(&bar, 0, &abort_flag, limit);
    if ((threadIdx.x & 31) == 0) gave_up[warp] = got ? 0 : 1;
}

// ---- vectors ----------------------------------------------------------------
__global__ void k_gather(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                         double *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}
__global__ void k_scatter(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ src,
                          double *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}
template <typename VT>
__global__ void k_set(int64_t n, VT *__restrict__ x, VT v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// y = A x (sub == 0) or y = b - A x (sub == 1); `lanes` threads per row.
// With zcol non-null, x is also copied into column ctl->j of zcol (leading
// dimension n): the FGMRES step stores z_j while it forms A z_j.
template <int LANES>
__global__ void __launch_bounds__(256)
k_spmv(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
       const double *__restrict__ v, const double *__restrict__ x, const double *__restrict__ b,
       double *__restrict__ y, double *__restrict__ zcol, const KrylovCtl *__restrict__ ctl) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = tid / LANES;
    const int sub = threadIdx.x % LANES;
    double acc = 0.0;
    if (row < n)
        for (int64_t p = rp[row] + sub; p < rp[row + 1]; p += LANES) acc += __ldg(v + p) * __ldg(x + __ldg(ci + p));
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, LANES);
    if (row < n && sub == 0) {
        y[row] = b ? b[row] - acc : acc;
        if (zcol) zcol[(int64_t)ctl->j * n + row] = x[row];
    }
}

// ---- Gram-Schmidt passes -------------------------------------------------------
// Every pass streams the rows [i0, i1) of one CTA once.  ncols <= kMaxCols.


__device__ __forceinline__ bool finish_block(unsigned *counter) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ void reduce_partials(const double *partial, int ncols1, double *out) {
    reduce_columns<double>(partial, (int)gridDim.x, ncols1, out);
}

// Partial dots of the NC columns V[:, c0 .. c0+NC) with w over the CTA's rows
// (and w . w into acc[NC] when WW).  The row loop issues every load of a row
// (two rows per iteration) before any arithmetic, so each thread keeps
// 2 (NC + 1) loads in flight: these passes are bound by memory latency and
// FP64 issue, not by bandwidth.  w is read through L2 (ld.global.cg): it may
// have been written earlier in the same kernel.
template <int NC, bool WW>
__device__ __forceinline__ void dots_group(const double *__restrict__ V, int64_t ldv, int c0, const double *w,
                                           int64_t i0, int64_t i1, double *acc) {
    const double *vc[NC > 0 ? NC : 1];
#pragma unroll
    for (int u = 0; u < NC; ++u) vc[u] = V + (int64_t)(c0 + u) * ldv;
    const int64_t st = blockDim.x;
    int64_t i = i0 + threadIdx.x;
    for (; i + st < i1; i += 2 * st) {
        const double wa = __ldcg(w + i), wb = __ldcg(w + i + st);
        double va[NC > 0 ? NC : 1], vb[NC > 0 ? NC : 1];
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            va[u] = vc[u][i];
            vb[u] = vc[u][i + st];
        }
#pragma unroll
        for (int u = 0; u < NC; ++u) acc[u] = fma(vb[u], wb, fma(va[u], wa, acc[u]));
        if (WW) acc[NC] = fma(wb, wb, fma(wa, wa, acc[NC]));
    }
    if (i < i1) {
        const double wa = __ldcg(w + i);
#pragma unroll
        for (int u = 0; u < NC; ++u) acc[u] = fma(vc[u][i], wa, acc[u]);
        if (WW) acc[NC] = fma(wa, wa, acc[NC]);
    }
}

// Block partial sums of V[:, c] . w for c < ncols and of w . w (slot ncols),
// written to partial[c * gridDim.x + blockIdx.x].  Columns go in groups of
// 8, 4, 2 and 1 (the group width is uniform, so the row loops have no
// branches), w . w with the first group.  The CTA reduction goes through
// shared memory (warp s sums slot s: eight values per lane, then one warp
// reduction), far fewer FP64 adds than full-warp butterflies per column.
// Requires blockDim.x == kReduceThreads.
__device__ void block_dots(const double *__restrict__ V, int64_t ldv, int ncols, const double *w,
                           int64_t i0, int64_t i1, double *partial) {
    static_assert(kReduceThreads % 32 == 0 && kReduceThreads / 32 >= 1, "whole warps");
    __shared__ double tred[9][kReduceThreads];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int c0 = 0;
    bool first = true;
    while (first || c0 < ncols) {
        const int rem = ncols - c0;
        const int nc = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : rem;
        double acc[9];
#pragma unroll
        for (int u = 0; u < 9; ++u) acc[u] = 0.0;
        switch (nc + (first ? 16 : 0)) {
            case 8: dots_group<8, false>(V, ldv, c0, w, i0, i1, acc); break;
            case 4: dots_group<4, false>(V, ldv, c0, w, i0, i1, acc); break;
            case 2: dots_group<2, false>(V, ldv, c0, w, i0, i1, acc); break;
            case 1: dots_group<1, false>(V, ldv, c0, w, i0, i1, acc); break;
            case 24: dots_group<8, true>(V, ldv, c0, w, i0, i1, acc); break;
            case 20: dots_group<4, true>(V, ldv, c0, w, i0, i1, acc); break;
            case 18: dots_group<2, true>(V, ldv, c0, w, i0, i1, acc); break;
            case 17: dots_group<1, true>(V, ldv, c0, w, i0, i1, acc); break;
            default: dots_group<0, true>(V, ldv, c0, w, i0, i1, acc); break;    // ncols == 0
        }
        const int ns = nc + (first ? 1 : 0);          // slots: nc columns, then w . w (in acc[nc])
#pragma unroll
        for (int u = 0; u < 9; ++u)
            if (u < ns) tred[u][threadIdx.x] = acc[u];
        __syncthreads();
        for (int sl = warp; sl < ns; sl += kReduceThreads / 32) {
            double sum = tred[sl][lane];
#pragma unroll
            for (int q = 1; q < kReduceThreads / 32; ++q) sum += tred[sl][q * 32 + lane];
            sum = warp_sum(sum);
            const int col = sl < nc ? c0 + sl : ncols;
            if (lane == 0) partial[(int64_t)col * gridDim.x + blockIdx.x] = sum;
        }
        __syncthreads();
        c0 += nc;
        first = false;
    }
}

// x_i - sum_c V[i, c] h_c, columns eight at a time with all eight loads
// issued first; hs must hold zeros from ncols up to the next multiple of 8
// (the padded slots load the last column again and multiply it by zero).
__device__ __forceinline__ double project_out(const double *__restrict__ V, int64_t ldv, int ncols,
                                              const double *hs, int64_t i, double x) {
    double a1 = 0.0;
    for (int c0 = 0; c0 < ncols; c0 += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = V[(int64_t)min(c0 + u, ncols - 1) * ldv + i];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            x = fma(-v[u], hs[c0 + u], x);
            a1 = fma(-v[u + 1], hs[c0 + u + 1], a1);
        }
    }
    return x + a1;
}

// project_out for the two rows ia and ib together: all sixteen loads of a
// column group are issued before its arithmetic.
__device__ __forceinline__ void project_pair(const double *__restrict__ V, int64_t ldv, int ncols, const double *hs,
                                             int64_t ia, int64_t ib, double &xa, double &xb) {
    double a1 = 0.0, b1 = 0.0;
    for (int c0 = 0; c0 < ncols; c0 += 8) {
        double va[8], vb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t off = (int64_t)min(c0 + u, ncols - 1) * ldv;
            va[u] = V[off + ia];
            vb[u] = V[off + ib];
        }
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            xa = fma(-va[u], hs[c0 + u], xa);
            a1 = fma(-va[u + 1], hs[c0 + u + 1], a1);
            xb = fma(-vb[u], hs[c0 + u], xb);
            b1 = fma(-vb[u + 1], hs[c0 + u + 1], b1);
        }
    }
    xa += a1;
    xb += b1;
}

// Sum of v over the CTA (kReduceThreads threads), valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kReduceThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kReduceThreads / 32; ++q) t += ws[q];
    }
    __syncthreads();
    return t;
}

// hs[c] = h[c] for c < ncols, zeros up to the next multiple of 8.
__device__ __forceinline__ void load_coefficients(double *hs, const double *h, int ncols) {
    const int np = (ncols + 7) & ~7;
    for (int c = threadIdx.x; c < np; c += blockDim.x) hs[c] = c < ncols ? __ldcg(h + c) : 0.0;
}

// Givens update of column j of the (m+1) x m Hessenberg matrix H (FGMRES).
__device__ void givens_step(KrylovCtl *ctl, double *H, double *cs, double *sn, double *g) {
    const int j = ctl->j, m1 = ctl->m + 1;
    double *h = H + (int64_t)j * m1;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    const double den = hypot(h[j], h[j + 1]);
    const double c = den == 0.0 ? 1.0 : h[j] / den;
    const double s = den == 0.0 ? 0.0 : h[j + 1] / den;
    cs[j] = c;
    sn[j] = s;
    h[j] = den;
    h[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    const double r = fabs(g[j + 1]);
    ctl->resid = r;
    ctl->iters += 1;
    ctl->jdone = j + 1;
    const bool bad = !isfinite(r) || !isfinite(den);
    if (bad) ctl->nonfinite = 1;
    if (r <= ctl->tol_abs || ctl->breakdown || bad || ctl->iters >= ctl->maxit || j + 1 >= ctl->m)
        ctl->stop = 1;
}

// After h (ncols values) and ||w||^2 are known: record h in column j of H and
// in hbuf (the projection coefficients of the next kernel: the Givens update
// below rotates the column of H in place), decide on a second pass and, if
// none, the norm of the projected vector.  Called by one whole warp: the
// stores and ||h||^2 are spread over its lanes, lane 0 takes the decisions.
__device__ void after_first_pass(KrylovCtl *ctl, const double *red, int ncols, double *H, double *cs,
                                 double *sn, double *g, double *hbuf) {
    const int lane = threadIdx.x & 31;
    const int j = ctl->j, m1 = ctl->m + 1;
    double hh = 0.0;
    for (int c = lane; c < ncols; c += 32) {
        H[(int64_t)j * m1 + c] = red[c];
        hbuf[c] = red[c];
        hh = fma(red[c], red[c], hh);
    }
    hh = warp_sum(hh);
    if (lane != 0) return;
    const double ww = red[ncols];
    ctl->wnorm2 = ww;
    const double rest = ww - hh;      // ||w - V h||^2 by Pythagoras
    const bool again = ctl->force_reorth || !(rest > 0.5 * ww);
    ctl->reorth = again ? 1 : 0;
    if (again) { ctl->nreorth += 1; return; }
    const double beta = sqrt(rest);
    ctl->beta = beta;
    ctl->breakdown = beta <= 1e-14 * sqrt(ww) ? 1 : 0;
    H[(int64_t)j * m1 + j + 1] = beta;
    if (ctl->givens) givens_step(ctl, H, cs, sn, g);
}

}  // namespace

// Pass 1: partial dots; finisher stores h, decides on reorthogonalisation.
// A step is only launched while its cycle is active (ctl->stop == 0).
__global__ void __launch_bounds__(kReduceThreads)
k_gs_dots(int64_t len, const double *__restrict__ V, int64_t ldv, const double *__restrict__ w,
          double *partial, unsigned *counter, KrylovCtl *ctl, double *H, double *cs, double *sn, double *g,
          double *hbuf) {
    if (ctl->stop) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->reorth = 0;
        return;
    }
    const int ncols = ctl->j + 1;
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    block_dots(V, ldv, ncols, w, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[kMaxCols + 1];
    reduce_partials(partial, ncols + 1, red);
    if (threadIdx.x < 32) after_first_pass(ctl, red, ncols, H, cs, sn, g, hbuf);
    if (threadIdx.x == 0) *counter = 0u;
}

// Pass 1 fused with the product that forms w: w = A z on the CTA's rows (one
// thread per row, CSR), z copied into column j of zcol (the FGMRES basis Z),
// then the same partial dots and finisher as k_gs_dots.  Every row of w is
// written and read back by the same thread, so no CTA-wide ordering is needed.
__global__ void __launch_bounds__(kReduceThreads)
k_gs_spmv_dots(int64_t len, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
               const double *__restrict__ av, const double *__restrict__ z, double *__restrict__ zcol,
               const double *__restrict__ V, int64_t ldv, double *w, double *partial, unsigned *counter,
               KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *hbuf) {
    if (ctl->stop) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->reorth = 0;
        return;
    }
    const int j = ctl->j, ncols = j + 1;
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    double *zj = zcol + (int64_t)j * len;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        // the first eight entries of the row with all index, value and x
        // loads in flight together (indices clamped into the row), the rest
        // (rows longer than eight) one by one
        const int64_t p0 = rp[i], p1 = rp[i + 1];
        double a0 = 0.0, a1 = 0.0;
        if (p1 > p0) {
            int cc[8];
            double vv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t pq = p0 + q < p1 ? p0 + q : p0;
                cc[q] = ci[pq];
                vv[q] = p0 + q < p1 ? av[pq] : 0.0;
            }
            double zz[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) zz[q] = z[cc[q]];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                a0 = fma(vv[q], zz[q], a0);
                a1 = fma(vv[q + 1], zz[q + 1], a1);
            }
            for (int64_t p = p0 + 8; p < p1; ++p) a0 = fma(av[p], z[ci[p]], a0);
        }
        w[i] = a0 + a1;
        zj[i] = z[i];
    }
    block_dots(V, ldv, ncols, w, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[kMaxCols + 1];
    reduce_partials(partial, ncols + 1, red);
    if (threadIdx.x < 32) after_first_pass(ctl, red, ncols, H, cs, sn, g, hbuf);
    if (threadIdx.x == 0) *counter = 0u;
}

// Pass 2: w -= V h with h from h2buf (the first-pass coefficients).  Without
// reorthogonalisation the result is scaled into V[:, j+1] (unless the step
// ended the cycle); otherwise w is kept, the second-pass coefficients h2 are
// reduced into h2buf (every CTA has read it by then) and added to H.
__global__ void __launch_bounds__(kReduceThreads)
k_gs_sub(int64_t len, double *__restrict__ V, int64_t ldv, double *__restrict__ w, double *partial,
         unsigned *counter, KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *h2buf,
         double *__restrict__ vcopy) {
    const int again = ctl->reorth;
    if (!again && (ctl->stop || ctl->breakdown)) return;
    __shared__ double hs[kMaxCols];
    const int j = ctl->j, ncols = j + 1, m1 = ctl->m + 1;
    load_coefficients(hs, h2buf, ncols);
    __syncthreads();
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    const double inv = again ? 0.0 : 1.0 / ctl->beta;
    double *vn = V + (int64_t)(j + 1) * ldv;
    const int64_t st = blockDim.x;
    int64_t i = i0 + threadIdx.x;
    for (; i + st < i1; i += 2 * st) {
        double xa = w[i], xb = w[i + st];
        project_pair(V, ldv, ncols, hs, i, i + st, xa, xb);
        if (again) {
            w[i] = xa;
            w[i + st] = xb;
        } else {
            vn[i] = xa * inv;
            vn[i + st] = xb * inv;
            if (vcopy) {
                vcopy[i] = xa * inv;
                vcopy[i + st] = xb * inv;
            }
        }
    }
    if (i < i1) {
        const double x = project_out(V, ldv, ncols, hs, i, w[i]);
        if (again) {
            w[i] = x;
        } else {
            vn[i] = x * inv;
            if (vcopy) vcopy[i] = x * inv;
        }
    }
    if (!again) return;
    __syncthreads();
    block_dots(V, ldv, ncols, w, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[kMaxCols + 1];
    reduce_partials(partial, ncols + 1, red);
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        H[(int64_t)j * m1 + c] += red[c];
        h2buf[c] = red[c];
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Pass 3 (only after a second Gram-Schmidt pass): w -= V h2 and an explicit
// ||w||^2 in the same sweep (Pythagoras would lose all accuracy to
// cancellation here); the finisher sets beta, the breakdown flag and the
// Givens update.
__global__ void __launch_bounds__(kReduceThreads)
k_gs_sub2(int64_t len, const double *__restrict__ V, int64_t ldv, double *__restrict__ w,
          const double *__restrict__ h2, double *partial, unsigned *counter, KrylovCtl *ctl, double *H, double *cs,
          double *sn, double *g) {
    if (!ctl->reorth) return;
    __shared__ double hs[kMaxCols];
    const int j = ctl->j, ncols = j + 1, m1 = ctl->m + 1;
    load_coefficients(hs, h2, ncols);
    __syncthreads();
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    // w -= V h2 and ||w||^2 in the same sweep
    double ww = 0.0;
    const int64_t st = blockDim.x;
    int64_t i = i0 + threadIdx.x;
    for (; i + st < i1; i += 2 * st) {
        double xa = w[i], xb = w[i + st];
        project_pair(V, ldv, ncols, hs, i, i + st, xa, xb);
        w[i] = xa;
        w[i + st] = xb;
        ww = fma(xb, xb, fma(xa, xa, ww));
    }
    if (i < i1) {
        const double x = project_out(V, ldv, ncols, hs, i, w[i]);
        w[i] = x;
        ww = fma(x, x, ww);
    }
    ww = block_sum(ww);
    if (threadIdx.x == 0) partial[blockIdx.x] = ww;
    if (!finish_block(counter)) return;
    __shared__ double red[1];
    reduce_partials(partial, 1, red);
    if (threadIdx.x == 0) {
        const double beta = sqrt(red[0]);
        ctl->beta = beta;
        ctl->breakdown = beta <= 1e-14 * sqrt(ctl->wnorm2) ? 1 : 0;
        H[(int64_t)j * m1 + j + 1] = beta;
        if (ctl->givens) givens_step(ctl, H, cs, sn, g);
        *counter = 0u;
    }
}

// After a second pass: V[:, j+1] = w / beta (and its copy), unless the cycle ended.
__global__ void k_gs_scale(int64_t len, double *__restrict__ V, int64_t ldv, const double *__restrict__ w,
                           const KrylovCtl *ctl, double *__restrict__ vcopy) {
    if (!ctl->reorth || ctl->stop || ctl->breakdown) return;
    __shared__ double sc;
    if (threadIdx.x == 0) sc = 1.0 / ctl->beta;               // once per CTA
    __syncthreads();
    const double inv = sc;
    double *vn = V + (int64_t)(ctl->j + 1) * ldv;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i] * inv;
        vn[i] = x;
        if (vcopy) vcopy[i] = x;
    }
}

// ---- FGMRES with delayed reorthogonalisation ------------------------------------------
// One reduction after each product.  The Krylov direction of step j, vt, is
// the first Gram-Schmidt pass of the previous product normalised by a
// Pythagorean estimate; its second pass (a = V^T vt, nu = ||vt - V a||) needs
// no product and is reduced beside M^{-1} (k_dgs_fix_adots, which also
// finalises the previous basis vector), and the reduction after the product
// gives, by linearity of M^{-1}, every coefficient of w = A M^{-1} vt against
// the final basis.  The stored preconditioned vectors Zt = M^{-1} vt relate to
// those of the final basis by an upper triangular R (Zt = Z R), so
// x = Zt R^{-1} y.  Column j-1 of the Hessenberg matrix is final at step j;
// the step's stopping test uses column j rotated provisionally.

// Final Givens step on column jc of Hrot (already rotated by 0..jc-1):
// rotation jc, g, residual estimate.  One reciprocal square root instead of
// hypot and two divisions: on this part a dependent FP64 operation costs on
// the order of a hundred cycles, so the finisher's critical path counts
// operations, not flops (the entries are O(||b||), far from overflow).
__device__ __forceinline__ double givens_close(double *col, int jc, double *cs, double *sn, double *g) {
    const double x = col[jc], y = col[jc + 1];
    const double q = fma(x, x, y * y);
    const double inv = q > 0.0 ? rsqrt(q) : 0.0;
    const double c = q > 0.0 ? x * inv : 1.0;
    const double s = q > 0.0 ? y * inv : 0.0;
    cs[jc] = c;
    sn[jc] = s;
    col[jc] = q * inv;
    col[jc + 1] = 0.0;
    g[jc + 1] = -s * g[jc];
    g[jc] = c * g[jc];
    return fabs(g[jc + 1]);
}

// Rotations 0..jc-1 (cs, sn) applied to col[0..jc] (shared memory) by one
// warp.  The carried entry obeys r_{i+1} = -s_i r_i + c_i col[i+1], an affine
// recurrence: every lane composes the maps of its contiguous segment, a
// shuffle scan combines the lanes (earlier segments first), and each lane then
// walks its segment from its prefix.  Dependent FP64 steps: about
// (jc / 32) + 2 log2(32) instead of 2 jc.
__device__ __forceinline__ void rotate_column_warp(const double *cs, const double *sn, int jc, double *col) {
    const int lane = threadIdx.x & 31;
    if (jc <= 0) return;
    const int per = (jc + 31) / 32;                 // <= 5 for kMaxCols
    const int lo = min(lane * per, jc), hi = min(lo + per, jc);
    double h[6], cc[5], ss[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int i = lo + q;
        cc[q] = i < hi ? cs[i] : 1.0;
        ss[q] = i < hi ? sn[i] : 0.0;
        h[q + 1] = i < hi ? col[i + 1] : 0.0;
    }
    const double h0 = col[0];
    __syncwarp();
    double A = 1.0, Bv = 0.0;                       // this segment's composed map
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if (lo + q < hi) {
            Bv = fma(-ss[q], Bv, cc[q] * h[q + 1]);
            A = -ss[q] * A;
        }
    double Ai = A, Bi = Bv;                         // inclusive scan over lanes
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double Ao = __shfl_up_sync(0xffffffffu, Ai, off), Bo = __shfl_up_sync(0xffffffffu, Bi, off);
        if (lane >= off) {
            Bi = fma(Ai, Bo, Bi);
            Ai = Ai * Ao;
        }
    }
    double Ae = __shfl_up_sync(0xffffffffu, Ai, 1), Be = __shfl_up_sync(0xffffffffu, Bi, 1);
    if (lane == 0) {
        Ae = 1.0;
        Be = 0.0;
    }
    double r = fma(Ae, h0, Be);                     // carried entry at the start of the segment
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if (lo + q < hi) {
            const double tq = fma(cc[q], r, ss[q] * h[q + 1]);
            r = fma(-ss[q], r, cc[q] * h[q + 1]);
            col[lo + q] = tq;
            if (lo + q == jc - 1) col[jc] = r;
        }
    __syncwarp();
}

// w[i] = (A z)_i and zj[i] = z[i] for the rows [i0, i1) of the CTA, two rows
// per thread and iteration: the row extents, then the first eight entries'
// columns and values, then the z values of both rows are each loaded together,
// so a thread waits for three memory round trips per pair of rows.  Entries
// past the eighth of a row (none for 7-point stencils) follow one by one.
// Returns the thread's share of w . vt.
__device__ __forceinline__ double spmv_rows_pair(int64_t i0, int64_t i1, const int64_t *__restrict__ rp,
                                                 const int32_t *__restrict__ ci, const double *__restrict__ av,
                                                 const double *__restrict__ z, double *__restrict__ w,
                                                 double *__restrict__ zj, const double *__restrict__ vt) {
    const int64_t st = blockDim.x;
    double dv = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 2 * st) {
        const int64_t ib = i + st;
        const bool hb = ib < i1;
        const int64_t pa0 = rp[i], pa1 = rp[i + 1];
        const int64_t pb0 = hb ? rp[ib] : pa0, pb1 = hb ? rp[ib + 1] : pa0;
        int ca[8], cb[8];
        double va[8], vb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            // absent entries read entry 0 of the matrix (always valid) with weight 0
            const int64_t qa = pa0 + q < pa1 ? pa0 + q : 0, qb = pb0 + q < pb1 ? pb0 + q : 0;
            ca[q] = ci[qa];
            cb[q] = ci[qb];
            va[q] = pa0 + q < pa1 ? av[qa] : 0.0;
            vb[q] = pb0 + q < pb1 ? av[qb] : 0.0;
        }
        double za[8], zb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            za[q] = z[ca[q]];
            zb[q] = z[cb[q]];
        }
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            a0 = fma(va[q], za[q], a0);
            a1 = fma(va[q + 1], za[q + 1], a1);
            b0 = fma(vb[q], zb[q], b0);
            b1 = fma(vb[q + 1], zb[q + 1], b1);
        }
        for (int64_t p = pa0 + 8; p < pa1; ++p) a0 = fma(av[p], z[ci[p]], a0);
        const double wa = a0 + a1;
        w[i] = wa;
        zj[i] = z[i];
        dv = fma(wa, vt[i], dv);
        if (hb) {
            for (int64_t p = pb0 + 8; p < pb1; ++p) b0 = fma(av[p], z[ci[p]], b0);
            const double wb = b0 + b1;
            w[ib] = wb;
            zj[ib] = z[ib];
            dv = fma(wb, vt[ib], dv);
        }
    }
    return dv;
}

// Step j: w = A z (z also stored in column j of Zt), then the reduction of
// V_{j-1}^T w, w . w and vt . w (V_{j-1}^T vt and vt . vt come from
// k_dgs_fix_adots, which ran beside M^{-1}); the finisher finalises column
// j-1, stores column j of R, forms the first-pass column h1 of step j, its
// lagged norm and the coefficients of the next direction, and decides whether
// the cycle ends.
__global__ void __launch_bounds__(kReduceThreads)
k_dgs_dots(int64_t len, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
           const double *__restrict__ av, const double *__restrict__ z, double *__restrict__ zcol,
           const double *__restrict__ V, int64_t ldv, const double *vt, double *w, double *partial, unsigned *counter,
           KrylovCtl *ctl, DgsBufs B) {
    if (ctl->stop) return;
    const int j = ctl->j;
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    double *zj = zcol + (int64_t)j * len;
    // w = A z with vt . w; V_{j-1}^T w and w . w (V_{j-1}^T vt and vt . vt were
    // formed beside M^{-1} by k_dgs_fix_adots): partial slots 0..j-1 V^T w,
    // j w . w, j+1 vt . w
    const double dv = block_sum(spmv_rows_pair(i0, i1, rp, ci, av, z, w, zj, vt));
    if (threadIdx.x == 0) partial[(int64_t)(j + 1) * gridDim.x + blockIdx.x] = dv;
    block_dots(V, ldv, j, w, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[2 * kMaxCols + 3];
    double *ash = red + kMaxCols + 2;
    for (int c = threadIdx.x; c < j; c += blockDim.x) ash[c] = __ldcg(B.apre + c);
    reduce_partials(partial, j + 2, red);
    // finisher: only what the next-direction sweep needs (a, V_j^T w, nu,
    // the lagged norm btil, the breakdown test); the Hessenberg column,
    // rotations and stopping test run beside that sweep (k_dgs_tail)
    __shared__ double sc[4];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const double *a = ash, *b = red;
    const double gam = ctl->gam_pre, om = red[j], dlt = red[j + 1];
    if (warp == 0) {
        double aa = 0.0, ab = 0.0;
        for (int c = lane; c < j; c += 32) {
            aa = fma(a[c], a[c], aa);
            ab = fma(a[c], b[c], ab);
        }
        aa = warp_sum(aa);
        ab = warp_sum(ab);
        if (lane == 0) {
            sc[0] = sqrt(fmax(gam - aa, 0.0));
            sc[1] = ab;
        }
    } else if (warp == 1) {
        double vv = 0.0;
        for (int c = lane; c < j; c += 32) vv = fma(b[c], b[c], vv);
        vv = warp_sum(vv);
        if (lane == 0) sc[2] = vv;
    }
    __syncthreads();
    const double nu = sc[0], inv_nu = 1.0 / nu;
    const double vjw = (dlt - sc[1]) * inv_nu;   // v_j . w
    for (int c = t; c < j; c += blockDim.x) {
        B.a[c] = a[c];
        B.coef[c] = b[c];
    }
    if (t != 0) return;
    B.coef[j] = vjw;
    const double rest = om - fma(vjw, vjw, sc[2]);  // ||w - V_j V_j^T w||^2 (Pythagoras)
    const double bt = rest > 0.0 ? sqrt(rest) * inv_nu : 0.0;
    const double w2 = om * inv_nu * inv_nu;
    ctl->btil_prev = ctl->btil;
    ctl->nu = nu;
    ctl->btil = bt;
    ctl->wnorm2 = w2;
    ctl->breakdown = bt <= 1e-14 * sqrt(fabs(w2)) ? 1 : 0;
    *counter = 0u;
}

// The rest of step j's finisher, one CTA of four warps on the second stream
// beside k_dgs_next (four warps of 64 registers fit beside seven CTAs of the
// sweep on one SM): column j-1 of the Hessenberg matrix is now final (rows
// 0..j-1 from the previous first pass plus the lagged correction, row j =
// btil_prev nu), and so is column j of R; the first-pass column of step j is
// h1 = (V_j^T w - Hraw[0..j, 0..j-1] a) / nu; rotations 0..j-2 act on both
// columns (one warp each), rotation j-1 closes column j-1, and the provisional
// rotation of column j gives the residual estimate that decides whether the
// cycle ends.  Nothing here is read by k_dgs_next.
__global__ void __launch_bounds__(128) k_dgs_tail(KrylovCtl *ctl, DgsBufs B) {
    __shared__ double s_cs[kMaxCols], s_sn[kMaxCols], s_g[kMaxCols + 1];
    __shared__ double hcol[kMaxCols + 1], h1s[kMaxCols + 2], s_a[kMaxCols], s_cf[kMaxCols + 1];
    if (ctl->stop) return;                          // no step ran (see k_dgs_dots)
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const int j = ctl->j;
    const int m1 = ctl->m + 1;
    const double nu = ctl->nu, inv_nu = 1.0 / nu, bprev = ctl->btil_prev, bt = ctl->btil;
    for (int c = t; c <= j; c += blockDim.x) {
        s_cs[c] = B.cs[c];
        s_sn[c] = B.sn[c];
        s_g[c] = B.g[c];
        s_cf[c] = __ldcg(B.coef + c);
        if (c < j) {
            const double ac = __ldcg(B.a + c);
            s_a[c] = ac;
            const double hv = B.hprev[c] + bprev * ac;
            hcol[c] = hv;
            B.Hraw[(int64_t)(j - 1) * m1 + c] = hv;
            B.R[c + (int64_t)j * m1] = ac;
        }
    }
    if (t == 0) {
        hcol[j] = bprev * nu;
        if (j > 0) B.Hraw[(int64_t)(j - 1) * m1 + j] = bprev * nu;
        B.R[j + (int64_t)j * m1] = nu;
    }
    __syncthreads();
    // g = Hraw[0..j, 0..j-1] a: columns before j-1 are final since earlier
    // steps (row r has entries in columns >= r-1), column j-1 is in hcol.  Warp
    // w takes rows w, w + nw, ... four at a time, its lanes the columns, so the
    // Hraw loads are issued together; the row sums go to h1s, which the loop
    // below overwrites row by row
    for (int rb = warp; rb <= j; rb += 4 * nw) {
        double acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = rb + u * nw;
            acc[u] = 0.0;
            if (r <= j)
                for (int c = (r > 0 ? r - 1 : 0) + lane; c < j - 1; c += 32)
                    acc[u] = fma(B.Hraw[(int64_t)c * m1 + r], s_a[c], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = warp_sum(acc[u]);
        if (lane == 0)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (rb + u * nw <= j) h1s[rb + u * nw] = acc[u];
    }
    __syncthreads();
    // the first-pass column h1 = (V_j^T w - g) / nu
    for (int r = t; r <= j; r += blockDim.x) {
        double g0 = h1s[r];
        if (j > 0) g0 = fma(hcol[r], s_a[j - 1], g0);
        const double h1 = (s_cf[r] - g0) * inv_nu;
        h1s[r] = h1;
        B.hprev[r] = h1;
    }
    __syncthreads();
    // rotations 0..j-2 on column j-1 (warp 0) and on column j (warp 1)
    if (warp == 0) rotate_column_warp(s_cs, s_sn, j - 1, hcol);
    else if (warp == 1) rotate_column_warp(s_cs, s_sn, j - 1, h1s);
    __syncthreads();
    if (t != 0) return;
    h1s[j + 1] = bt;
    if (j > 0) {
        givens_close(hcol, j - 1, s_cs, s_sn, s_g);
        B.cs[j - 1] = s_cs[j - 1];
        B.sn[j - 1] = s_sn[j - 1];
        B.g[j - 1] = s_g[j - 1];
        B.g[j] = s_g[j];
        for (int i = 0; i <= j; ++i) B.Hrot[(int64_t)(j - 1) * m1 + i] = hcol[i];
        const double c = s_cs[j - 1], s = s_sn[j - 1];      // rotation j-1 on column j
        const double tt = c * h1s[j - 1] + s * h1s[j];
        h1s[j] = -s * h1s[j - 1] + c * h1s[j];
        h1s[j - 1] = tt;
    }
    const double qd = fma(h1s[j], h1s[j], h1s[j + 1] * h1s[j + 1]);
    const double prelim = qd > 0.0 ? fabs(h1s[j + 1] * rsqrt(qd) * s_g[j]) : 0.0;
    ctl->resid = prelim;
    ctl->iters += 1;
    const bool bad = !isfinite(prelim) || !isfinite(nu) || !isfinite(bt);
    if (bad) ctl->nonfinite = 1;
    if (prelim <= ctl->tol_abs || ctl->breakdown || bad || ctl->iters >= ctl->maxit || j + 1 >= ctl->m) ctl->stop = 1;
}

// Sum over the first nc columns of V at row i of V[i, c] * h[c] (h in shared
// memory), columns eight at a time and the rest in groups of 4, 2 and 1, every
// load of a group issued before its arithmetic (nc is uniform over the grid).
__device__ __forceinline__ double combine_row(const double *__restrict__ V, int64_t ldv, int nc, const double *h,
                                              int64_t i) {
    double x = 0.0, y = 0.0;
    int c0 = 0;
    for (; c0 + 8 <= nc; c0 += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = V[(int64_t)(c0 + u) * ldv + i];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            x = fma(v[u], h[c0 + u], x);
            y = fma(v[u + 1], h[c0 + u + 1], y);
        }
    }
    if (c0 + 4 <= nc) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = V[(int64_t)(c0 + u) * ldv + i];
        x = fma(v[0], h[c0], x);
        y = fma(v[1], h[c0 + 1], y);
        x = fma(v[2], h[c0 + 2], x);
        y = fma(v[3], h[c0 + 3], y);
        c0 += 4;
    }
    if (c0 + 2 <= nc) {
        const double v0 = V[(int64_t)c0 * ldv + i], v1 = V[(int64_t)(c0 + 1) * ldv + i];
        x = fma(v0, h[c0], x);
        y = fma(v1, h[c0 + 1], y);
        c0 += 2;
    }
    if (c0 < nc) x = fma(V[(int64_t)c0 * ldv + i], h[c0], x);
    return x + y;
}

// Step j, second sweep (the part the next application of M^{-1} waits for):
// with v_j = (vt_j - V_{j-1} a) / nu, the next direction
//   vt_{j+1} = (w - V_{j-1} coef[0..j) - v_j coef[j]) / (nu btil)
//            = (w - V_{j-1} (coef[0..j) - a coef[j] / nu) - vt_j coef[j] / nu) / (nu btil)
// needs one pass over V_{j-1} and not v_j itself; vt_{j+1} replaces vt_j in
// place (not after a breakdown) and vt_j is kept in V[:, j] until k_dgs_fix
// reorthogonalises it.
__global__ void __launch_bounds__(256)
k_dgs_next(int64_t len, double *__restrict__ V, int64_t ldv, double *vt, const double *__restrict__ w,
           const KrylovCtl *ctl, DgsBufs B) {
    __shared__ double cf[kMaxCols];
    __shared__ double sc[2];
    const int j = ctl->j;
    const bool next = !ctl->breakdown && ctl->btil > 0.0;
    // the step's scalars once per CTA: an FP64 division is a long sequence on
    // the slow FP64 pipe, and this grid has a thread per row
    if (threadIdx.x == 0) {
        const double nu = ctl->nu, inv_nu = 1.0 / nu;
        sc[0] = __ldcg(B.coef + j) * inv_nu;
        sc[1] = next ? inv_nu / ctl->btil : 0.0;
    }
    __syncthreads();
    const double cj = sc[0];
    for (int c = threadIdx.x; c < j; c += blockDim.x) cf[c] = fma(-__ldcg(B.a + c), cj, __ldcg(B.coef + c));
    __syncthreads();
    const double inv_nb = sc[1];
    double *vj = V + (int64_t)j * ldv;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += st) {
        const double x = combine_row(V, ldv, j, cf, i);
        const double t = __ldcg(vt + i);
        vj[i] = t;
        if (next) vt[i] = fma(-t, cj, w[i] - x) * inv_nb;
    }
}

// Beside z = M^{-1} vt_j (second stream, SMs the substitutions leave free):
// the previous step's reorthogonalisation v_{j-1} = (vt_{j-1} - V_{j-2} a) / nu
// (as k_dgs_fix), then a = V_{j-1}^T vt_j and vt_j . vt_j, which do not need
// M^{-1}: into B.apre and ctl->gam_pre.  The fixed column's dot is formed from
// the value just computed (register), the other columns by block_dots.
// Partial slots: 0..j-2 V_{j-2}^T vt, j-1 vt . vt (j = 0: slot 0), j v_{j-1} . vt.
__global__ void __launch_bounds__(kReduceThreads)
k_dgs_fix_adots(int64_t len, double *V, int64_t ldv, const double *vt, double *partial, unsigned *counter,
                KrylovCtl *ctl, DgsBufs B) {
    __shared__ double as[kMaxCols];
    const int j = ctl->j, jp = j - 1;
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    double dv = 0.0;
    if (jp >= 0) {
        for (int c = threadIdx.x; c < jp; c += blockDim.x) as[c] = __ldcg(B.a + c);
        __syncthreads();
        const double inv_nu = 1.0 / ctl->nu;
        double *vj = V + (int64_t)jp * ldv;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double v = (vj[i] - combine_row(V, ldv, jp, as, i)) * inv_nu;
            vj[i] = v;
            dv = fma(v, vt[i], dv);
        }
    }
    dv = block_sum(dv);
    if (jp >= 0 && threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = dv;
    const int nc = jp > 0 ? jp : 0;
    block_dots(V, ldv, nc, vt, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[kMaxCols + 2];
    reduce_partials(partial, jp >= 0 ? j + 1 : 1, red);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) B.apre[c] = red[c];
    if (threadIdx.x == 0) {
        if (jp >= 0) B.apre[jp] = red[j];
        ctl->gam_pre = red[nc];
        *counter = 0u;
    }
}

// The reorthogonalisation of step jp = ctl->j + off, off the critical path:
// V[:, jp] = (vt_jp - V_{jp-1} a) / nu, with a and nu of step jp (the next
// step's reduction overwrites them only after this kernel; the FGMRES step
// runs it beside the next application of M^{-1}).  Nothing for jp < 0.
__global__ void __launch_bounds__(256)
k_dgs_fix(int64_t len, double *__restrict__ V, int64_t ldv, const KrylovCtl *ctl, DgsBufs B, int off) {
    __shared__ double as[kMaxCols];
    __shared__ double sc;
    const int jp = ctl->j + off;
    if (jp < 0) return;
    for (int c = threadIdx.x; c < jp; c += blockDim.x) as[c] = __ldcg(B.a + c);
    if (threadIdx.x == 0) sc = 1.0 / ctl->nu;                 // once per CTA (a thread per row)
    __syncthreads();
    const double inv_nu = sc;
    double *vj = V + (int64_t)jp * ldv;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += st)
        vj[i] = (vj[i] - combine_row(V, ldv, jp, as, i)) * inv_nu;
}

// End of a cycle: the reduction of the last direction against V_j finalises
// column j (after a breakdown the direction is not formed: a = 0, h_{j+1,j} =
// 0); final rotation of column j, jdone = j + 1.
__global__ void __launch_bounds__(kReduceThreads)
k_dgs_close(int64_t len, const double *__restrict__ V, int64_t ldv, const double *vt, double *partial,
            unsigned *counter, KrylovCtl *ctl, DgsBufs B) {
    const int j = ctl->j;
    const bool brk = ctl->breakdown || !(ctl->btil > 0.0);
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    if (!brk) block_dots(V, ldv, j + 1, vt, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[kMaxCols + 1];
    if (!brk) reduce_partials(partial, j + 2, red);
    __shared__ double s_cs[kMaxCols], s_sn[kMaxCols], s_g[kMaxCols + 1], col[kMaxCols + 2], sc[1];
    const int t = threadIdx.x, lane = t & 31, m1 = ctl->m + 1;
    for (int c = t; c <= j; c += blockDim.x) {
        s_cs[c] = B.cs[c];
        s_sn[c] = B.sn[c];
        s_g[c] = B.g[c];
    }
    if (t < 32) {
        double aa = 0.0;
        if (!brk)
            for (int c = lane; c <= j; c += 32) aa = fma(red[c], red[c], aa);
        aa = warp_sum(aa);
        if (lane == 0) sc[0] = brk ? 0.0 : sqrt(fmax(red[j + 1] - aa, 0.0));
    }
    __syncthreads();
    const double nu = sc[0];
    const double bt = brk ? 0.0 : ctl->btil;
    for (int c = t; c <= j; c += blockDim.x) {
        const double hv = B.hprev[c] + (brk ? 0.0 : bt * red[c]);
        col[c] = hv;
        B.Hraw[(int64_t)j * m1 + c] = hv;
    }
    if (t == 0) {
        col[j + 1] = bt * nu;
        B.Hraw[(int64_t)j * m1 + j + 1] = bt * nu;
    }
    __syncthreads();
    if (t < 32) rotate_column_warp(s_cs, s_sn, j, col);
    __syncthreads();
    if (t != 0) return;
    const double r = givens_close(col, j, s_cs, s_sn, s_g);
    B.cs[j] = s_cs[j];
    B.sn[j] = s_sn[j];
    B.g[j] = s_g[j];
    B.g[j + 1] = s_g[j + 1];
    for (int i = 0; i <= j + 1; ++i) B.Hrot[(int64_t)j * m1 + i] = col[i];
    ctl->resid = r;
    ctl->jdone = j + 1;
    if (!isfinite(r)) ctl->nonfinite = 1;
    *counter = 0u;
}

// y = Hrot^{-1} g over the first jdone columns, then (R != nullptr) y = R^{-1} y;
// column-oriented back substitutions, one CTA (the updates of a column in
// parallel, one dependent step per column).
__global__ void __launch_bounds__(256)
k_lsq2(const KrylovCtl *ctl, const double *__restrict__ H, const double *__restrict__ g, const double *R,
       double *__restrict__ y) {
    __shared__ double s[kMaxCols];
    const int jd = ctl->jdone, m1 = ctl->m + 1;
    for (int i = threadIdx.x; i < jd; i += blockDim.x) s[i] = g[i];
    __syncthreads();
    for (int pass = 0; pass < (R ? 2 : 1); ++pass) {
        const double *T = pass == 0 ? H : R;
        for (int i = jd - 1; i >= 0; --i) {
            const double yi = s[i] / T[(int64_t)i * m1 + i];
            for (int r = threadIdx.x; r < i; r += blockDim.x) s[r] = fma(-T[(int64_t)i * m1 + r], yi, s[r]);
            __syncthreads();
            if (threadIdx.x == 0) s[i] = yi;
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < jd; i += blockDim.x) y[i] = s[i];
}

// Advance to the next column (one thread).
__global__ void k_gs_next(KrylovCtl *ctl) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !ctl->stop) ctl->j += 1;
}

// ||x||^2 into *out (partials + finisher).
__global__ void __launch_bounds__(kReduceThreads)
k_norm2(int64_t len, const double *__restrict__ x, double *partial, unsigned *counter, double *out) {
    const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min((int64_t)blockIdx.x * chunk, len), i1 = min(i0 + chunk, len);
    block_dots(x, 0, 0, x, i0, i1, partial);
    if (!finish_block(counter)) return;
    __shared__ double red[1];
    reduce_partials(partial, 1, red);
    if (threadIdx.x == 0) { *out = red[0]; *counter = 0u; }
}

// v = x * (1 / sqrt(*n2))
__global__ void k_scale_by_norm(int64_t len, const double *__restrict__ x, const double *n2, double *__restrict__ v,
                                double *__restrict__ vcopy) {
    __shared__ double sc;
    if (threadIdx.x == 0) sc = 1.0 / sqrt(*n2);               // once per CTA
    __syncthreads();
    const double inv = sc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        v[i] = x[i] * inv;
        if (vcopy) vcopy[i] = x[i] * inv;
    }
}

// Start of an FGMRES cycle: g = (beta, 0, ...), j = 0 (one thread).
__global__ void k_cycle_start(KrylovCtl *ctl, double *g, const double *n2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= ctl->m; ++i) g[i] = 0.0;
    g[0] = sqrt(*n2);
    ctl->j = 0;
    ctl->stop = 0;
    ctl->breakdown = 0;
    ctl->reorth = 0;
    ctl->jdone = 0;
}

// y = R^{-1} g (back substitution on the rotated Hessenberg), one thread.
__global__ void k_lsq(const KrylovCtl *ctl, const double *H, const double *g, double *y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int jd = ctl->jdone, m1 = ctl->m + 1;
    for (int i = jd - 1; i >= 0; --i) {
        double s = g[i];
        for (int t = i + 1; t < jd; ++t) s -= H[(int64_t)t * m1 + i] * y[t];
        y[i] = s / H[(int64_t)i * m1 + i];
    }
}

// x += Z[:, :jdone] y
__global__ void k_update_x(int64_t len, const double *__restrict__ Z, int64_t ldz, const KrylovCtl *ctl,
                           const double *__restrict__ y, double *__restrict__ x) {
    __shared__ double ys[kMaxCols];
    const int jd = ctl->jdone;
    for (int c = threadIdx.x; c < jd; c += blockDim.x) ys[c] = y[c];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = x[i];
        for (int c = 0; c < jd; ++c) acc += Z[(int64_t)c * ldz + i] * ys[c];
        x[i] = acc;
    }
}

// out[:, c] = V[:, :mm] Q[:, c] for c < kk (thick restart of the Arnoldi basis).
__global__ void k_basis_rotate(int64_t len, const double *__restrict__ V, int64_t ldv, int mm,
                               const double *__restrict__ Q, int kk, double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < kk; ++c) {
            double acc = 0.0;
            for (int d = 0; d < mm; ++d) acc += V[(int64_t)d * ldv + i] * Q[d + (int64_t)c * mm];
            out[(int64_t)c * ldv + i] = acc;
        }
    }
}

// ---- graph-resident FGMRES control (conditional WHILE nodes) ----------------------
// Cycle start inside the outer loop body: g = (||r||, 0, ...), j = 0, and the
// inner loop's condition set so that the first Arnoldi step runs.
__global__ void k_cycle_start_g(KrylovCtl *ctl, double *g, const double *n2, cudaGraphConditionalHandle inner) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= ctl->m; ++i) g[i] = 0.0;
    g[0] = sqrt(*n2);
    ctl->j = 0;
    ctl->stop = 0;
    ctl->breakdown = 0;
    ctl->reorth = 0;
    ctl->jdone = 0;
    cudaGraphSetConditional(inner, 1u);
}

// End of one Arnoldi step: advance j, continue while the cycle is active.
__global__ void k_step_end_g(KrylovCtl *ctl, cudaGraphConditionalHandle inner) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!ctl->stop) ctl->j += 1;
    cudaGraphSetConditional(inner, ctl->stop ? 0u : 1u);
}

// End of a cycle: true residual test (Sec. 5 set-up), restart or finish.
__global__ void k_cycle_end_g(KrylovCtl *ctl, const double *n2r, cudaGraphConditionalHandle outer) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double rn = sqrt(*n2r);
    ctl->rnorm = rn;
    bool again = true;
    if (!isfinite(rn) || ctl->nonfinite) {
        ctl->nonfinite = 1;
        again = false;
    } else if (rn <= ctl->tol_abs) {
        ctl->converged = 1;
        again = false;
    } else if (ctl->iters >= ctl->maxit) {
        again = false;
    } else {
        ctl->restarts += 1;
    }
    cudaGraphSetConditional(outer, again ? 1u : 0u);
}

// ---- host launchers -----------------------------------------------------------------
static int grid_for(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)(g > cap ? cap : g);
}

template <typename VT, typename WT>
void launch_trsv(const LevelView<VT, WT> &lv, int mode, int smem_rows, const IoT<VT> *in, VT *work,
                 IoT<VT> *out_final, VT *scratch, cudaStream_t st, const PendingLowRank<VT, WT> &pl) {
    if (lv.nblk == 0) return;
    const bool smem = smem_rows > 0;
    const size_t bytes = kRingBytes + (smem ? (size_t)smem_rows * sizeof(VT) : 0);
    // FP32: register slots sized to the level's longest row (4, 8, 12 or 16)
    const int ne = LanesPerRow<VT>::value != 1 ? 16 : lv.max_slots <= 4 ? 4 : lv.max_slots <= 8 ? 8
                                                 : lv.max_slots <= 12 ? 12 : 16;
#define GEMSLR_TRSV(M, S, N) \
    k_trsv<VT, WT, M, S, N><<<lv.nblk, kTrsvThreads2, bytes, st>>>(lv, in, work, out_final, scratch, pl)
#define GEMSLR_TRSV_NE(M, S)                  \
    switch (ne) {                             \
        case 4: GEMSLR_TRSV(M, S, 4); break;  \
        case 8: GEMSLR_TRSV(M, S, 8); break;  \
        case 12: GEMSLR_TRSV(M, S, 12); break; \
        default: GEMSLR_TRSV(M, S, 16); break; \
    }
    if constexpr (LanesPerRow<VT>::value == 1) {
        if (mode == 0) {
            if (smem) { GEMSLR_TRSV_NE(0, true) }
            else { GEMSLR_TRSV_NE(0, false) }
        } else {
            if (smem) { GEMSLR_TRSV_NE(1, true) }
            else { GEMSLR_TRSV_NE(1, false) }
        }
    } else {
        if (mode == 0) {
            if (smem) GEMSLR_TRSV(0, true, 16);
            else GEMSLR_TRSV(0, false, 16);
        } else {
            if (smem) GEMSLR_TRSV(1, true, 16);
            else GEMSLR_TRSV(1, false, 16);
        }
    }
#undef GEMSLR_TRSV_NE
#undef GEMSLR_TRSV
    count_launch();
}

template <typename VT, typename WT>
void set_trsv_smem_limit(int bytes) {
    auto set = [&](auto fn, int b) { cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b); };
    set(k_trsv<VT, WT, 0, true, 16>, bytes);
    set(k_trsv<VT, WT, 1, true, 16>, bytes);
    set(k_trsv<VT, WT, 0, false, 16>, kRingBytes);
    set(k_trsv<VT, WT, 1, false, 16>, kRingBytes);
    if constexpr (LanesPerRow<VT>::value == 1) {
        set(k_trsv<VT, WT, 0, true, 4>, bytes);
        set(k_trsv<VT, WT, 0, true, 8>, bytes);
        set(k_trsv<VT, WT, 0, true, 12>, bytes);
        set(k_trsv<VT, WT, 1, true, 4>, bytes);
        set(k_trsv<VT, WT, 1, true, 8>, bytes);
        set(k_trsv<VT, WT, 1, true, 12>, bytes);
        set(k_trsv<VT, WT, 0, false, 4>, kRingBytes);
        set(k_trsv<VT, WT, 0, false, 8>, kRingBytes);
        set(k_trsv<VT, WT, 0, false, 12>, kRingBytes);
        set(k_trsv<VT, WT, 1, false, 4>, kRingBytes);
        set(k_trsv<VT, WT, 1, false, 8>, kRingBytes);
        set(k_trsv<VT, WT, 1, false, 12>, kRingBytes);
    }
}

template <typename VT, typename WT>
void launch_couple(const LevelView<VT, WT> &lv, const IoT<VT> *in, VT *work, VT *partial, unsigned *counter,
                   VT *u, cudaStream_t st, const PendingLowRank<VT, WT> &pl) {
    if (lv.stail == 0) return;
    const int grid = (int)((lv.stail + kCoupleRows - 1) / kCoupleRows);
    k_couple<VT, WT><<<grid, kCoupleRows, 0, st>>>(lv, in, work, partial, counter, u, pl); count_launch();
}


template void launch_trsv<double, double>(const LevelView<double, double> &, int, int, const double *, double *,
                                          double *, double *, cudaStream_t, const PendingLowRank<double, double> &);
template void launch_trsv<float, __nv_bfloat16>(const LevelView<float, __nv_bfloat16> &, int, int, const double *,
                                                float *, double *, float *, cudaStream_t,
                                                const PendingLowRank<float, __nv_bfloat16> &);
template void launch_trsv<zc, zc>(const LevelView<zc, zc> &, int, int, const zc *, zc *, zc *, zc *, cudaStream_t,
                                  const PendingLowRank<zc, zc> &);
template void set_trsv_smem_limit<double, double>(int);
template void set_trsv_smem_limit<zc, zc>(int);
template void set_trsv_smem_limit<float, __nv_bfloat16>(int);
template void launch_couple<double, double>(const LevelView<double, double> &, const double *, double *, double *,
                                            unsigned *, double *, cudaStream_t,
                                            const PendingLowRank<double, double> &);
template void launch_couple<zc, zc>(const LevelView<zc, zc> &, const zc *, zc *, zc *, unsigned *, zc *, cudaStream_t,
                                    const PendingLowRank<zc, zc> &);
template void launch_couple<float, __nv_bfloat16>(const LevelView<float, __nv_bfloat16> &, const double *, float *,
                                                  float *, unsigned *, float *, cudaStream_t,
                                                  const PendingLowRank<float, __nv_bfloat16> &);

void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t st) {
    if (n > 0) { k_gather<<<grid_for(n, 256, 4864), 256, 0, st>>>(n, perm, src, dst); count_launch(); }
}
void launch_scatter(int64_t n, const int32_t *perm, const double *src, double *dst, cudaStream_t st) {
    if (n > 0) { k_scatter<<<grid_for(n, 256, 4864), 256, 0, st>>>(n, perm, src, dst); count_launch(); }
}
void launch_zero(int64_t n, double *x, cudaStream_t st) {
    if (n > 0) { k_set<double><<<grid_for(n, 256, 4864), 256, 0, st>>>(n, x, 0.0); count_launch(); }
}
void launch_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x,
                 const double *b, double *y, int lanes, cudaStream_t st, double *zcol, const KrylovCtl *ctl) {
    if (n == 0) return;
    const int64_t threads = n * lanes;
    const int grid = (int)((threads + 255) / 256);
    switch (lanes) {
        case 2: k_spmv<2><<<grid, 256, 0, st>>>(n, rp, ci, v, x, b, y, zcol, ctl); break;
        case 4: k_spmv<4><<<grid, 256, 0, st>>>(n, rp, ci, v, x, b, y, zcol, ctl); break;
        case 16: k_spmv<16><<<grid, 256, 0, st>>>(n, rp, ci, v, x, b, y, zcol, ctl); break;
        default: k_spmv<8><<<grid, 256, 0, st>>>(n, rp, ci, v, x, b, y, zcol, ctl); break;
    }
    count_launch();
}
void launch_gs_dots(int64_t len, const double *V, int64_t ldv, const double *w, double *partial, unsigned *counter,
                    KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *hbuf, int grid,
                    cudaStream_t st) {
    k_gs_dots<<<grid, kReduceThreads, 0, st>>>(len, V, ldv, w, partial, counter, ctl, H, cs, sn, g, hbuf);
    count_launch();
}
void launch_gs_spmv_dots(int64_t len, const int64_t *rp, const int32_t *ci, const double *av, const double *z,
                         double *zcol, const double *V, int64_t ldv, double *w, double *partial, unsigned *counter,
                         KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *hbuf, int grid,
                         cudaStream_t st) {
    k_gs_spmv_dots<<<grid, kReduceThreads, 0, st>>>(len, rp, ci, av, z, zcol, V, ldv, w, partial, counter, ctl, H, cs,
                                                     sn, g, hbuf);
    count_launch();
}
void launch_gs_sub(int64_t len, double *V, int64_t ldv, double *w, double *partial, unsigned *counter,
                   KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, double *h2buf, int grid,
                   cudaStream_t st, double *vcopy) {
    k_gs_sub<<<grid, kReduceThreads, 0, st>>>(len, V, ldv, w, partial, counter, ctl, H, cs, sn, g, h2buf, vcopy);
    count_launch();
}
void launch_gs_sub2(int64_t len, double *V, int64_t ldv, double *w, const double *h2, double *partial,
                    unsigned *counter, KrylovCtl *ctl, double *H, double *cs, double *sn, double *g, int grid,
                    cudaStream_t st) {
    k_gs_sub2<<<grid, kReduceThreads, 0, st>>>(len, V, ldv, w, h2, partial, counter, ctl, H, cs, sn, g);
    count_launch();
}
void launch_gs_scale(int64_t len, double *V, int64_t ldv, const double *w, const KrylovCtl *ctl, double *vcopy,
                     cudaStream_t st) {
    k_gs_scale<<<grid_for(len, 256, 1216), 256, 0, st>>>(len, V, ldv, w, ctl, vcopy);
    count_launch();
}
void launch_wait_selftest(long long limit, int32_t *gave_up, cudaStream_t st) {
    k_wait_selftest<<<1, 64, 0, st>>>(limit, gave_up);
    count_launch();
}
void launch_dgs_dots(int64_t len, const int64_t *rp, const int32_t *ci, const double *av, const double *z, double *zcol,
                     const double *V, int64_t ldv, const double *vt, double *w, double *partial, unsigned *counter,
                     KrylovCtl *ctl, const DgsBufs &B, int grid, cudaStream_t st) {
    k_dgs_dots<<<grid, kReduceThreads, 0, st>>>(len, rp, ci, av, z, zcol, V, ldv, vt, w, partial, counter, ctl, B);
    count_launch();
}
void launch_dgs_next(int64_t len, double *V, int64_t ldv, double *vt, const double *w, const KrylovCtl *ctl,
                     const DgsBufs &B, cudaStream_t st) {
    k_dgs_next<<<grid_for(len, 256, 1216), 256, 0, st>>>(len, V, ldv, vt, w, ctl, B);
    count_launch();
}
constexpr int kFixExclusiveSmem = 170 * 1024;
void launch_dgs_fix(int64_t len, double *V, int64_t ldv, const KrylovCtl *ctl, const DgsBufs &B, int off, int grid,
                    bool exclusive, cudaStream_t st) {
    // exclusive: each CTA reserves more shared memory than an SM has left
    // beside any substitution CTA (>= 66 KB), so the two never share an SM
    // and the latency-bound substitutions keep theirs to themselves
    k_dgs_fix<<<grid, 256, exclusive ? kFixExclusiveSmem : 0, st>>>(len, V, ldv, ctl, B, off);
    count_launch();
}
void launch_dgs_fix_adots(int64_t len, double *V, int64_t ldv, const double *vt, double *partial, unsigned *counter,
                          KrylovCtl *ctl, const DgsBufs &B, int grid, cudaStream_t st) {
    // exclusive: see launch_dgs_fix
    k_dgs_fix_adots<<<grid, kReduceThreads, kFixExclusiveSmem, st>>>(len, V, ldv, vt, partial, counter, ctl, B);
    count_launch();
}
void launch_dgs_tail(KrylovCtl *ctl, const DgsBufs &B, cudaStream_t st) {
    k_dgs_tail<<<1, 128, 0, st>>>(ctl, B);
    count_launch();
}
void prepare_krylov_kernels() {
    GEMSLR_CUDA(cudaFuncSetAttribute(k_dgs_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, kFixExclusiveSmem));
    GEMSLR_CUDA(cudaFuncSetAttribute(k_dgs_fix_adots, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kFixExclusiveSmem));
}
void launch_dgs_close(int64_t len, const double *V, int64_t ldv, const double *vt, double *partial, unsigned *counter,
                      KrylovCtl *ctl, const DgsBufs &B, int grid, cudaStream_t st) {
    k_dgs_close<<<grid, kReduceThreads, 0, st>>>(len, V, ldv, vt, partial, counter, ctl, B);
    count_launch();
}
void launch_lsq2(const KrylovCtl *ctl, const double *H, const double *g, const double *R, double *y, cudaStream_t st) {
    k_lsq2<<<1, 256, 0, st>>>(ctl, H, g, R, y);
    count_launch();
}
void launch_gs_next(KrylovCtl *ctl, cudaStream_t st) { k_gs_next<<<1, 32, 0, st>>>(ctl); count_launch(); }
void launch_norm2(int64_t len, const double *x, double *partial, unsigned *counter, double *out, int grid,
                  cudaStream_t st) {
    k_norm2<<<grid, kReduceThreads, 0, st>>>(len, x, partial, counter, out); count_launch();
}
void launch_scale_by_norm(int64_t len, const double *x, const double *n2, double *v, cudaStream_t st, double *vcopy) {
    if (len > 0) { k_scale_by_norm<<<grid_for(len, 256, 4864), 256, 0, st>>>(len, x, n2, v, vcopy); count_launch(); }
}
void launch_cycle_start(KrylovCtl *ctl, double *g, const double *n2, cudaStream_t st) {
    k_cycle_start<<<1, 32, 0, st>>>(ctl, g, n2); count_launch();
}
void launch_lsq(const KrylovCtl *ctl, const double *H, const double *g, double *y, cudaStream_t st) {
    k_lsq<<<1, 32, 0, st>>>(ctl, H, g, y); count_launch();
}
void launch_update_x(int64_t len, const double *Z, int64_t ldz, const KrylovCtl *ctl, const double *y, double *x,
                     cudaStream_t st) {
    if (len > 0) { k_update_x<<<grid_for(len, 256, 4864), 256, 0, st>>>(len, Z, ldz, ctl, y, x); count_launch(); }
}
void launch_basis_rotate(int64_t len, const double *V, int64_t ldv, int mm, const double *Q, int kk, double *out,
                         cudaStream_t st) {
    if (len > 0) { k_basis_rotate<<<grid_for(len, 256, 4864), 256, 0, st>>>(len, V, ldv, mm, Q, kk, out); count_launch(); }
}

}  // namespace gemslr

namespace gemslr {
void launch_cycle_start_g(KrylovCtl *ctl, double *g, const double *n2, cudaGraphConditionalHandle h, cudaStream_t st) {
    k_cycle_start_g<<<1, 32, 0, st>>>(ctl, g, n2, h);
    count_launch();
}
void launch_step_end_g(KrylovCtl *ctl, cudaGraphConditionalHandle h, cudaStream_t st) {
    k_step_end_g<<<1, 32, 0, st>>>(ctl, h);
    count_launch();
}
void launch_cycle_end_g(KrylovCtl *ctl, const double *n2r, cudaGraphConditionalHandle h, cudaStream_t st) {
    k_cycle_end_g<<<1, 32, 0, st>>>(ctl, n2r, h);
    count_launch();
}
}  // namespace gemslr
