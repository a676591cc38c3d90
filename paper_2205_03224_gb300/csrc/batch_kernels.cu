// Batched kernels: many independent GeMSLR systems, kBatchRhs right-hand
// sides each, one launch per stage of M^{-1} (Alg. 2) over every system, and
// FGMRES (Sec. 4.1) run for every (system, rhs) pair in lock step.
// Preconditioner in FP32 (W in BF16, FP32 accumulation), Krylov in FP64.
#include "batch.cuh"
#include "device.h"
#include "ptx.cuh"

namespace gemslr {

namespace {
constexpr int R8 = kBatchRhs;

// Named barrier 1 over the consumer warps of the batched substitutions.
__device__ __forceinline__ void batch_consumer_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kBatchWarps) : "memory");
}

__device__ __forceinline__ bool last_of(unsigned *counter, unsigned n) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == n - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}
}  // namespace

// ---- M^{-1} stages -------------------------------------------------------------------
// Level-scheduled substitutions over the blocks of every system.  A block's
// right-hand sides are split over kBatchRhs / RPC CTAs of RPC each, so that
// the block's vector (rows x RPC) fits in shared memory: CTA c works on block
// c / (kBatchRhs / RPC), right-hand sides RPC * (c % (kBatchRhs / RPC)) on.
// The lanes of a warp are up to 4 rows x RPC right-hand sides.  MODE 0:
// right-hand side from `in` (FP64) or `work`.  MODE 1: right-hand side F y2,
// then work[rows] -= result.  Without SMEM (blocks too large even for RPC = 1)
// RPC is kBatchRhs and the vector stays in global memory.
template <int MODE, bool SMEM, int RPC>
__global__ void __launch_bounds__(kBatchTrsvThreads)
k_btrsv(const BatchLevel lv, const double *__restrict__ in, float *__restrict__ work, double *__restrict__ out_final,
        float *__restrict__ scratch) {
    static_assert(SMEM || RPC == R8, "the global-memory path keeps all right-hand sides");
    constexpr int kSplit = R8 / RPC;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *ring = smem;
    constexpr int CPG = 1, kSlots = kRingData / kStageBytes;   // the warps share every chunk: one per copy
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kRingData);
    uint64_t *empty = full + kSlots;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + kSlots + 1);
    float *xs_smem = reinterpret_cast<float *>(smem + kRingBytes);
    const int b = lv.order[blockIdx.x / kSplit];
    if (lv.live && !lv.live[lv.blk_sys[b]]) return;          // the whole CTA
    const int rhs0 = RPC * (blockIdx.x % kSplit);
    const int64_t r0 = lv.blk_r0[b];
    const int nr = lv.blk_nr[b];
    if (nr == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = lv.C.blk_chunk[b], c1 = lv.C.blk_chunk[b + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CPG * kBatchWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == kBatchWarps) {
        produce_chunks<CPG>(lv.C.data, lv.C.off, c0, c1, ring, full, empty, abort_flag, lv.err, lane);
        return;
    }
    const int ct = threadIdx.x;
    constexpr int NC = 32 * kBatchWarps;
    float *mine = work + r0 * R8;
    float *xs = SMEM ? xs_smem : (MODE == 1 ? scratch + lv.blk_f0[b] * R8 : mine);
    const int64_t f0 = lv.blk_f0[b];
    for (int idx = ct; idx < nr * RPC; idx += NC) {
        const int i = idx / RPC, r = rhs0 + idx % RPC;
        if (MODE == 1) {
            float acc = 0.f;
            for (int64_t p = lv.F_rp[f0 + i]; p < lv.F_rp[f0 + i + 1]; ++p) acc += lv.F_v[p] * work[(int64_t)lv.F_ci[p] * R8 + r];
            xs[idx] = acc;
        } else if (in) {
            xs[idx] = (float)in[(r0 + i) * R8 + r];
        } else if (SMEM) {
            xs[idx] = mine[i * R8 + r];
        }
    }
    batch_consumer_barrier();
    bool aborted = false;
    const int rr = lane / RPC, r = lane % RPC;
    const unsigned char *base = nullptr;
    for (int c = c0; c < c1; ++c) {
        const int k = c - c0;
        base = aborted ? nullptr : next_chunk<float, CPG>(ring, full, abort_flag, k, base);
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
            const int ne = S * nrow;
            const float *vals = reinterpret_cast<const float *>(cols + ((ne + 3) & ~3));
            const float *dinv = vals + ((ne + 3) & ~3);
            const int per = (nrow + kBatchWarps - 1) / kBatchWarps;   // <= 4 rows per warp
            const int t = warp * per + rr;
            if (rr < per && t < nrow) {
                const int row = rows[t], len = lens[t];
                // stored values are -t_ij (L) and -u_ij/u_ii (U): x_row d + sum v x,
                // x_row's load overlapping the chains
                const float self = xs[row * RPC + r], d = upper ? dinv[t] : 1.f;
                float a0 = 0.f, a1 = 0.f;
                int q = 0;
                for (; q + 1 < len; q += 2) {
                    a0 += vals[q * nrow + t] * xs[cols[q * nrow + t] * RPC + r];
                    a1 += vals[(q + 1) * nrow + t] * xs[cols[(q + 1) * nrow + t] * RPC + r];
                }
                if (q < len) a0 += vals[q * nrow + t] * xs[cols[q * nrow + t] * RPC + r];
                xs[row * RPC + r] = fmaf(self, d, a0 + a1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[chunk_slot<CPG>(k)]);
        }
        batch_consumer_barrier();
    }
    batch_consumer_barrier();
    if (*abort_flag) {
        if (ct == 0) atomicExch(lv.err, 1);
        return;
    }
    for (int idx = ct; idx < nr * RPC; idx += NC) {
        const int64_t g = (int64_t)(idx / RPC) * R8 + rhs0 + idx % RPC;
        float y = xs[idx];
        if (MODE == 1) y = mine[g] - y;
        // down: z1 (in place already without SMEM); up: the lower levels' up
        // sweeps gather this level's result from work, nothing reads the first level's
        const bool keep = MODE == 0 ? SMEM : !(lv.final_up && out_final);
        if (keep) mine[g] = y;
        if (out_final) out_final[r0 * R8 + g] = (double)y;
    }
}

// ---- BF16 tensor-core products with W (mma.sync m16n8k16, FP32 accumulation) ----------
// The 8 right-hand sides are the n = 8 of the tile.  W is stored in BF16; the
// FP32 vector operand is split into two BF16 terms v = hi + lo (hi = bf16(v),
// lo = bf16(v - hi)), so that each product carries about 16 significant bits
// of the vector (relative error ~2^-16) and W's own BF16 rounding is the only
// reduced-precision step, as in the CUDA-core path.
__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x (low 16 bits) = lo_elem
    return *reinterpret_cast<const uint32_t *>(&p);
}
__device__ __forceinline__ void split_bf16(float v, float &hi, float &lo) {
    hi = __bfloat162float(__float2bfloat16_rn(v));
    lo = v - hi;
}
// D (16 x 8, FP32) += A (16 x 16, BF16, row-major fragment) * B (16 x 8, BF16, column-major fragment).
__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// Fragment coordinates of m16n8k16 for lane = 4 * g + t (g = group 0..7, t = 0..3):
//   A: a[0] rows g, cols 2t, 2t+1; a[1] rows g+8, cols 2t, 2t+1; a[2] row g, cols 2t+8, 2t+9;
//      a[3] row g+8, cols 2t+8, 2t+9 (lower column in the low 16 bits);
//   B: b[0] rows (k) 2t, 2t+1, col (n) g; b[1] rows 2t+8, 2t+9, col g;
//   D: d[0], d[1] row g, cols 2t, 2t+1; d[2], d[3] row g+8, cols 2t, 2t+1.
// B fragments (hi and lo) of a K-slice [kk, kk+16) of a row-major k x 8 FP32
// matrix in shared memory (rows past kmax are zero).
__device__ __forceinline__ void b_frag_split(const float *M8, int kk, int kmax, int lane, uint32_t bh[2],
                                             uint32_t bl[2]) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r0 = kk + 2 * t + 8 * h, r1 = r0 + 1;
        const float v0 = r0 < kmax ? M8[r0 * R8 + g] : 0.f, v1 = r1 < kmax ? M8[r1 * R8 + g] : 0.f;
        float h0, l0, h1, l1;
        split_bf16(v0, h0, l0);
        split_bf16(v1, h1, l1);
        bh[h] = pack_bf16(h0, h1);
        bl[h] = pack_bf16(l0, l1);
    }
}

// z2 = b2 - E z1 on the CTA's tail rows, partial W_s^T z2 (tensor cores), and
// (last CTA of the system) u_s = H_s (W_s^T z2).
__global__ void __launch_bounds__(kBatchThreads)
k_bcouple(const BatchLevel lv, const double *__restrict__ in, float *__restrict__ work) {
    __shared__ float zs[256 * R8];
    __shared__ float ts[kBatchMaxRank * R8];
    __shared__ float half2[kBatchMaxRank * R8];
    const int c = blockIdx.x, s = lv.cta_seg[c];
    if (lv.live && !lv.live[s]) return;                       // every CTA of the system
    const int64_t i0 = lv.cta_i0[c], len = lv.seg_len[s];
    const int rows = (int)min((int64_t)lv.rows_cta, len - i0);
    const int64_t g0 = lv.seg_r0[s] + i0, e0 = lv.seg_e0[s] + i0;
    for (int idx = threadIdx.x; idx < rows * R8; idx += blockDim.x) {
        const int i = idx / R8, r = idx % R8;
        const int64_t g = g0 + i;
        float z = in ? (float)in[g * R8 + r] : work[g * R8 + r];
        for (int64_t p = lv.E_rp[e0 + i]; p < lv.E_rp[e0 + i + 1]; ++p) z -= lv.E_v[p] * work[(int64_t)lv.E_ci[p] * R8 + r];
        work[g * R8 + r] = z;
        zs[idx] = z;
    }
    const int k = lv.seg_k[s];
    if (k == 0) return;
    __syncthreads();
    // partial W^T z: M = columns of W (16 per tile), K = the CTA's rows, N = 8 rhs.
    // Warp w takes column tile w % 4 and every other K-slice (parity w / 4).
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *Ws = lv.W + lv.seg_w0[s];
    const int mt = warp & 3, par = warp >> 2;
    const int ntile = (k + 15) / 16;
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    if (mt < ntile) {
        const int ca = 16 * mt + g, cb = ca + 8;          // the two W columns of this lane's A rows
        const __nv_bfloat16 z16 = __float2bfloat16_rn(0.f);
        for (int kk = 16 * par; kk < rows; kk += 32) {
            uint32_t a[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {                 // h = 0: K cols 2t, 2t+1; h = 1: + 8
                const int i = kk + 2 * t + 8 * h;
                const __nv_bfloat16 wa0 = (ca < k && i < rows) ? Ws[(int64_t)ca * len + i0 + i] : z16;
                const __nv_bfloat16 wa1 = (ca < k && i + 1 < rows) ? Ws[(int64_t)ca * len + i0 + i + 1] : z16;
                const __nv_bfloat16 wb0 = (cb < k && i < rows) ? Ws[(int64_t)cb * len + i0 + i] : z16;
                const __nv_bfloat16 wb1 = (cb < k && i + 1 < rows) ? Ws[(int64_t)cb * len + i0 + i + 1] : z16;
                a[2 * h] = (uint32_t)__bfloat16_as_ushort(wa0) | ((uint32_t)__bfloat16_as_ushort(wa1) << 16);
                a[2 * h + 1] = (uint32_t)__bfloat16_as_ushort(wb0) | ((uint32_t)__bfloat16_as_ushort(wb1) << 16);
            }
            uint32_t bh[2], bl[2];
            b_frag_split(zs, kk, rows, lane, bh, bl);
            mma_bf16_16816(d, a, bh);
            mma_bf16_16816(d, a, bl);
        }
    }
    // the two K-parities of a column tile are added in a fixed order
    if (par == 1 && mt < ntile) {
        half2[(16 * mt + g) * R8 + 2 * t] = d[0];
        half2[(16 * mt + g) * R8 + 2 * t + 1] = d[1];
        half2[(16 * mt + g + 8) * R8 + 2 * t] = d[2];
        half2[(16 * mt + g + 8) * R8 + 2 * t + 1] = d[3];
    }
    __syncthreads();
    if (par == 0 && mt < ntile) {
        const int rr[4] = {16 * mt + g, 16 * mt + g, 16 * mt + g + 8, 16 * mt + g + 8};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cc = rr[q], col = 2 * t + (q & 1);
            if (cc < k) lv.partial[((int64_t)c * kBatchMaxRank + cc) * R8 + col] = d[q] + half2[cc * R8 + col];
        }
    }
    const int ca = lv.seg_cta0[s], cb = lv.seg_cta0[s + 1];
    if (!last_of(&lv.seg_counter[s], (unsigned)(cb - ca))) return;
    for (int idx = threadIdx.x; idx < k * R8; idx += blockDim.x) {
        const int cc = idx / R8, rr = idx % R8;
        float acc = 0.f;
        for (int q = ca; q < cb; ++q) acc += __ldcg(lv.partial + ((int64_t)q * kBatchMaxRank + cc) * R8 + rr);
        ts[idx] = acc;
    }
    __syncthreads();
    const float *Hs = lv.H + lv.seg_h0[s];
    for (int idx = threadIdx.x; idx < k * R8; idx += blockDim.x) {
        const int cc = idx / R8, rr = idx % R8;
        float acc = 0.f;
        for (int d2 = 0; d2 < k; ++d2) acc += Hs[cc + (int64_t)d2 * k] * ts[d2 * R8 + rr];
        lv.u[((int64_t)s * kBatchMaxRank + cc) * R8 + rr] = acc;
    }
    if (threadIdx.x == 0) lv.seg_counter[s] = 0u;
}

// work[tail] += W_s u_s (tensor cores: M = 16 tail rows per tile, K = the rank,
// N = 8 rhs; each warp takes every eighth row tile).
__global__ void __launch_bounds__(kBatchThreads)
k_blowrank(const BatchLevel lv, float *__restrict__ work) {
    __shared__ float us[kBatchMaxRank * R8];
    const int c = blockIdx.x, s = lv.cta_seg[c];
    const int k = lv.seg_k[s];
    if (k == 0 || (lv.live && !lv.live[s])) return;
    const int64_t i0 = lv.cta_i0[c], len = lv.seg_len[s];
    const int rows = (int)min((int64_t)lv.rows_cta, len - i0);
    for (int idx = threadIdx.x; idx < k * R8; idx += blockDim.x) us[idx] = lv.u[(int64_t)s * kBatchMaxRank * R8 + idx];
    __syncthreads();
    const __nv_bfloat16 *Ws = lv.W + lv.seg_w0[s];
    const int64_t g0 = lv.seg_r0[s] + i0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 z16 = __float2bfloat16_rn(0.f);
    for (int rt = warp; 16 * rt < rows; rt += nw) {
        const int ra = 16 * rt + g, rb = ra + 8;          // this lane's two A rows
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kk = 0; kk < k; kk += 16) {
            uint32_t a[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {                 // K cols 2t, 2t+1 (+ 8 for h = 1)
                const int cc = kk + 2 * t + 8 * h;
                const __nv_bfloat16 wa0 = (ra < rows && cc < k) ? Ws[(int64_t)cc * len + i0 + ra] : z16;
                const __nv_bfloat16 wa1 = (ra < rows && cc + 1 < k) ? Ws[(int64_t)(cc + 1) * len + i0 + ra] : z16;
                const __nv_bfloat16 wb0 = (rb < rows && cc < k) ? Ws[(int64_t)cc * len + i0 + rb] : z16;
                const __nv_bfloat16 wb1 = (rb < rows && cc + 1 < k) ? Ws[(int64_t)(cc + 1) * len + i0 + rb] : z16;
                a[2 * h] = (uint32_t)__bfloat16_as_ushort(wa0) | ((uint32_t)__bfloat16_as_ushort(wa1) << 16);
                a[2 * h + 1] = (uint32_t)__bfloat16_as_ushort(wb0) | ((uint32_t)__bfloat16_as_ushort(wb1) << 16);
            }
            uint32_t bh[2], bl[2];
            b_frag_split(us, kk, k, lane, bh, bl);
            mma_bf16_16816(d, a, bh);
            mma_bf16_16816(d, a, bl);
        }
        if (ra < rows) {
            work[(g0 + ra) * R8 + 2 * t] += d[0];
            work[(g0 + ra) * R8 + 2 * t + 1] += d[1];
        }
        if (rb < rows) {
            work[(g0 + rb) * R8 + 2 * t] += d[2];
            work[(g0 + rb) * R8 + 2 * t + 1] += d[3];
        }
    }
}

// ---- Krylov kernels (FP64, per (system, rhs) pair) ---------------------------------

// y = A x or y = b - A x over the batch (block-diagonal A, batch columns);
// zcol: copy x into column *j of zcol (leading dimension ld).
__global__ void __launch_bounds__(256)
k_bspmv(int64_t nrows, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
        const double *__restrict__ x, const double *__restrict__ b, double *__restrict__ y, double *__restrict__ zcol,
        const int32_t *__restrict__ jp, int64_t ld, const int32_t *__restrict__ sys_of,
        const int32_t *__restrict__ live) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * R8) return;
    const int64_t g = idx / R8;
    if (live && !live[sys_of[g]]) return;      // every pair of the system has stopped
    const int r = (int)(idx % R8);
    double acc = 0.0;
    for (int64_t p = rp[g]; p < rp[g + 1]; ++p) acc += v[p] * x[(int64_t)ci[p] * R8 + r];
    y[idx] = b ? b[idx] - acc : acc;
    if (zcol) zcol[(int64_t)(*jp) * ld + idx] = x[idx];
}

namespace {
// Per-CTA partial dot products of columns 0..ncols-1 of V (and of w itself
// when with_norm) with w over rows [r0, r1), for the 8 right-hand sides.
// Threads: r = tid & 7, row group = tid >> 3 (32 groups); 4 columns at a time.
// w may have been written earlier in the same kernel, so it is read through L2.
__device__ void bdots_block(const double *__restrict__ V, int64_t ldv, int ncols, bool with_norm,
                            const double *w, int64_t r0, int64_t r1, double *partial_cta) {
    __shared__ double red[8][4][R8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int r = threadIdx.x & 7, grp = threadIdx.x >> 3;
    const int ntot = ncols + (with_norm ? 1 : 0);
    for (int c0 = 0; c0 < ntot; c0 += 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t g = r0 + grp; g < r1; g += 32) {
            const double wi = __ldcg(w + g * R8 + r);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + u;
                if (c < ncols) acc[u] += V[(int64_t)c * ldv + g * R8 + r] * wi;
                else if (c < ntot) acc[u] += wi * wi;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            double x = acc[u];
            x += __shfl_xor_sync(0xffffffffu, x, 8);
            x += __shfl_xor_sync(0xffffffffu, x, 16);
            if (lane < 8) red[warp][u][r] = x;
        }
        __syncthreads();
        if (threadIdx.x < 4 * R8) {
            const int u = threadIdx.x / R8, rr = threadIdx.x % R8, c = c0 + u;
            if (c < ntot) {
                double sum = 0.0;
                for (int q = 0; q < nw; ++q) sum += red[q][u][rr];
                partial_cta[c * R8 + rr] = sum;
            }
        }
        __syncthreads();
    }
}

// Sum the partials of system s's CTAs: out[c * 8 + r].
__device__ void bdots_finish(const double *partial, int ca, int cb, int ntot, double *out) {
    for (int idx = threadIdx.x; idx < ntot * R8; idx += blockDim.x) {
        double sum = 0.0;
        for (int q = ca; q < cb; ++q) sum += __ldcg(partial + (int64_t)q * (kMaxCols + 1) * R8 + idx);
        out[idx] = sum;
    }
    __syncthreads();
}

// Givens update of column j of pair p's Hessenberg matrix (as in the single-system solver).
__device__ void bgivens(const BatchKrylov &K, int p, int j) {
    const int m = K.m, m1 = m + 1;
    double *h = K.H + (int64_t)p * m1 * m + (int64_t)j * m1;
    double *cs = K.cs + (int64_t)p * (m + 2), *sn = K.sn + (int64_t)p * (m + 2), *g = K.g + (int64_t)p * (m + 2);
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    const double den = hypot(h[j], h[j + 1]);
    const double c = den == 0.0 ? 1.0 : h[j] / den, s = den == 0.0 ? 0.0 : h[j + 1] / den;
    cs[j] = c;
    sn[j] = s;
    const double brk = h[j + 1];
    h[j] = den;
    h[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    const double rsd = fabs(g[j + 1]);
    K.resid[p] = rsd;
    K.jdone[p] = j + 1;
    const bool bad = !isfinite(rsd) || !isfinite(den);
    if (bad) K.bad[p] = 1;
    const bool breakdown = brk <= 1e-14 * sqrt(K.wn2[p]);
    if (rsd <= K.tol[p] || breakdown || bad || *K.iters + j + 1 >= *K.maxit || j + 1 >= m) K.run[p] = 0;
}
}  // namespace

// The dot products of a Gram-Schmidt pass, h = V^T w: one thread per (column,
// rhs, row class) item streams over all rows of the CTA with register
// accumulators (the items of a row share its w through L1), so that no
// barrier interrupts the loads; the CTA's item sums go to its partials, and
// the system's last CTA finishes the pass.  Pass 1 stores h1; pass 2 (after
// w -= V h1 by k_bgs_sub) adds h2 to the Hessenberg column.  Every pass keeps
// its coefficients in hbuf for the subtraction that follows it.
constexpr int kGs1Threads = 512;

template <int PASS>
__global__ void __launch_bounds__(kGs1Threads)
k_bgs_dots(const BatchSegs S, BatchKrylov K, const double *__restrict__ V, int64_t ldv,
           const double *__restrict__ w) {
    extern __shared__ __align__(16) double acc[];   // max(8 (m + 1), kGs1Threads) item sums
    const int c = blockIdx.x, s = S.cta_sys[c];
    if (!K.sys_run[s]) return;                  // every CTA of the system
    const int64_t r0 = S.cta_r0[c], r1 = S.cta_r1[c];
    const int j = *K.j, ncols = j + 1;
    const int t = threadIdx.x;
    const int npairs = ncols * R8;
    const int rs = npairs >= kGs1Threads ? 1 : kGs1Threads / npairs;   // row classes per pair
    const int items = npairs * rs;
    for (int q = t; q < items; q += kGs1Threads) {
        const int pr = q % npairs, part = q / npairs, rr = pr & 7;
        const double *vp = V + (int64_t)(pr >> 3) * ldv + rr;
        const double *wp = w + rr;
        double a0 = 0.0, a1 = 0.0;
        int64_t g = r0 + part;
        for (; g + rs < r1; g += 2 * rs) {
            a0 += vp[g * R8] * wp[g * R8];
            a1 += vp[(g + rs) * R8] * wp[(g + rs) * R8];
        }
        if (g < r1) a0 += vp[g * R8] * wp[g * R8];
        acc[q] = a0 + a1;
    }
    __syncthreads();
    double *part_out = K.partial + (int64_t)c * (kMaxCols + 1) * R8;
    for (int pr = t; pr < npairs; pr += kGs1Threads) {
        double sum = 0.0;
        for (int p2 = 0; p2 < rs; ++p2) sum += acc[pr + p2 * npairs];
        part_out[pr] = sum;
    }
    const int ca = S.sys_cta0[s], cb = S.sys_cta0[s + 1];
    if (!last_of(&S.sys_counter[s], (unsigned)(cb - ca))) return;
    double *out = acc;                          // ncols x R8 sums of the system
    bdots_finish(K.partial, ca, cb, ncols, out);
    if (t < R8) {
        const int p = s * R8 + t, m1 = K.m + 1;
        double *hcol = K.H + (int64_t)p * m1 * K.m + (int64_t)j * m1;
        if (K.run[p]) {
            for (int cc = 0; cc < ncols; ++cc) {
                const double h = out[cc * R8 + t];
                if (PASS == 1) hcol[cc] = h;
                else hcol[cc] += h;
                K.hbuf[(int64_t)p * kMaxCols + cc] = h;
            }
        } else if (PASS == 2) {
            for (int cc = 0; cc < ncols; ++cc) K.hbuf[(int64_t)p * kMaxCols + cc] = 0.0;
            K.beta[p] = 0.0;
        }
    }
    if (t == 0) S.sys_counter[s] = 0u;
}

// w -= V h (h = the coefficients of the pass before, kept per pair in hbuf).
__global__ void __launch_bounds__(256)
k_bgs_sub(const BatchSegs S, BatchKrylov K, const double *__restrict__ V, int64_t ldv, double *__restrict__ w) {
    __shared__ double hs[R8][kMaxCols + 1];      // odd row stride: the 8 rhs of a warp in 8 banks
    const int c = blockIdx.x, s = S.cta_sys[c];
    if (!K.sys_run[s]) return;
    const int64_t r0 = S.cta_r0[c], r1 = S.cta_r1[c];
    const int ncols = *K.j + 1;
    for (int idx = threadIdx.x; idx < R8 * ncols; idx += blockDim.x) {
        const int rr = idx / ncols, cc = idx % ncols;
        hs[rr][cc] = K.hbuf[(int64_t)(s * R8 + rr) * kMaxCols + cc];
    }
    __syncthreads();
    const int rr = threadIdx.x & 7;             // r0 * 8 and the stride are multiples of 8
    for (int64_t idx = r0 * R8 + threadIdx.x; idx < r1 * R8; idx += blockDim.x) {
        double x0 = w[idx], x1 = 0.0;
        int cc = 0;
        for (; cc + 1 < ncols; cc += 2) {
            x0 -= V[(int64_t)cc * ldv + idx] * hs[rr][cc];
            x1 -= V[(int64_t)(cc + 1) * ldv + idx] * hs[rr][cc + 1];
        }
        if (cc < ncols) x0 -= V[(int64_t)cc * ldv + idx] * hs[rr][cc];
        w[idx] = x0 + x1;
    }
}

// w -= V h2 with ||w_p||^2 summed on the way (an explicit norm: Pythagoras
// would lose all accuracy to cancellation after the second pass); the
// per-system finisher sets beta_p and the pair's Givens update.
__global__ void __launch_bounds__(256)
k_bgs_subnorm(const BatchSegs S, BatchKrylov K, const double *__restrict__ V, int64_t ldv, double *__restrict__ w) {
    __shared__ double hs[R8][kMaxCols + 1];      // odd row stride: the 8 rhs of a warp in 8 banks
    __shared__ double red[8][R8];
    __shared__ double out[R8];
    const int c = blockIdx.x, s = S.cta_sys[c];
    if (!K.sys_run[s]) return;
    const int64_t r0 = S.cta_r0[c], r1 = S.cta_r1[c];
    const int j = *K.j, ncols = j + 1;
    for (int idx = threadIdx.x; idx < R8 * ncols; idx += blockDim.x) {
        const int rr = idx / ncols, cc = idx % ncols;
        hs[rr][cc] = K.hbuf[(int64_t)(s * R8 + rr) * kMaxCols + cc];
    }
    __syncthreads();
    const int rr = threadIdx.x & 7;             // r0 * 8 and the stride are multiples of 8
    double sq = 0.0;
    for (int64_t idx = r0 * R8 + threadIdx.x; idx < r1 * R8; idx += blockDim.x) {
        double x0 = w[idx], x1 = 0.0;
        int cc = 0;
        for (; cc + 1 < ncols; cc += 2) {
            x0 -= V[(int64_t)cc * ldv + idx] * hs[rr][cc];
            x1 -= V[(int64_t)(cc + 1) * ldv + idx] * hs[rr][cc + 1];
        }
        if (cc < ncols) x0 -= V[(int64_t)cc * ldv + idx] * hs[rr][cc];
        const double x = x0 + x1;
        w[idx] = x;
        sq += x * x;
    }
    sq += __shfl_xor_sync(0xffffffffu, sq, 8);
    sq += __shfl_xor_sync(0xffffffffu, sq, 16);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < R8) red[warp][lane] = sq;
    __syncthreads();
    if (threadIdx.x < R8) {
        double sum = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[q][threadIdx.x];
        K.partial[(int64_t)c * (kMaxCols + 1) * R8 + threadIdx.x] = sum;
    }
    const int ca = S.sys_cta0[s], cb = S.sys_cta0[s + 1];
    if (!last_of(&S.sys_counter[s], (unsigned)(cb - ca))) return;
    bdots_finish(K.partial, ca, cb, 1, out);
    if (threadIdx.x < R8) {
        const int rr = threadIdx.x, p = s * R8 + rr;
        const int m1 = K.m + 1;
        double *hcol = K.H + (int64_t)p * m1 * K.m + (int64_t)j * m1;
        if (K.run[p]) {
            const double beta = sqrt(out[rr]);
            double htot = 0.0;
            for (int cc = 0; cc < ncols; ++cc) htot += hcol[cc] * hcol[cc];
            K.wn2[p] = htot + beta * beta;          // ||A z_j||^2
            K.beta[p] = beta;
            hcol[j + 1] = beta;
            bgivens(K, p, j);
        } else {
            K.beta[p] = 0.0;
        }
    }
    if (threadIdx.x == 0) S.sys_counter[s] = 0u;
}

// V[:, j+1] = w / beta for pairs still running (0 otherwise); vin = same.
__global__ void __launch_bounds__(256)
k_bgs_final(const BatchSegs S, BatchKrylov K, double *__restrict__ V, int64_t ldv, const double *__restrict__ w,
            double *__restrict__ vin) {
    __shared__ double inv[R8];
    const int c = blockIdx.x, s = S.cta_sys[c];
    if (!K.sys_run[s]) return;
    const int64_t r0 = S.cta_r0[c], r1 = S.cta_r1[c];
    const int j = *K.j;
    if (threadIdx.x < R8) {
        const int p = s * R8 + threadIdx.x;
        inv[threadIdx.x] = (K.run[p] && K.beta[p] > 0.0) ? 1.0 / K.beta[p] : 0.0;
    }
    __syncthreads();
    double *vn = V + (int64_t)(j + 1) * ldv;
    for (int64_t idx = r0 * R8 + threadIdx.x; idx < r1 * R8; idx += blockDim.x) {
        const double v = w[idx] * inv[idx % R8];
        vn[idx] = v;
        vin[idx] = v;
    }
}

// ||x_p||^2 for every pair into out[p].
__global__ void __launch_bounds__(256)
k_bnorm2(const BatchSegs S, double *partial, const double *__restrict__ x, double *out) {
    __shared__ double o[R8 * (kMaxCols + 1)];
    const int c = blockIdx.x, s = S.cta_sys[c];
    bdots_block(nullptr, 0, 0, true, x, S.cta_r0[c], S.cta_r1[c], partial + (int64_t)c * (kMaxCols + 1) * R8);
    const int ca = S.sys_cta0[s], cb = S.sys_cta0[s + 1];
    if (!last_of(&S.sys_counter[s], (unsigned)(cb - ca))) return;
    bdots_finish(partial, ca, cb, 1, o);
    if (threadIdx.x < R8) out[s * R8 + threadIdx.x] = o[threadIdx.x];
    if (threadIdx.x == 0) S.sys_counter[s] = 0u;
}

// Before the first cycle: pair tolerances and states from ||b_p||^2 (in rn2).
__global__ void k_binit(BatchKrylov K, double rtol, int maxit) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < K.npair; p += gridDim.x * blockDim.x) {
        const double bn2 = K.rn2[p];
        const bool fin = isfinite(bn2);
        K.tol[p] = rtol * sqrt(fin ? bn2 : 0.0);
        K.active[p] = (fin && bn2 > 0.0) ? 1 : 0;
        K.conv[p] = (fin && bn2 == 0.0) ? 1 : 0;
        K.bad[p] = fin ? 0 : 1;
        K.its[p] = 0;
        K.restarts[p] = 0;
        K.run[p] = 0;
        K.jdone[p] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *K.iters = 0;
        *K.maxit = maxit;
        *K.j = 0;
    }
}

// Cycle start: g_p = (||r_p||, 0, ...), pairs still active run; V[:,0] = r_p / ||r_p||.
// sys_run[s] = some pair of system s still steps (one block; K.run final).
__device__ void sys_flags(const BatchKrylov &K) {
    for (int s = threadIdx.x; s < K.npair / R8; s += blockDim.x) {
        int any = 0;
        for (int r = 0; r < R8; ++r) any |= K.run[s * R8 + r];
        K.sys_run[s] = any;
    }
}

__global__ void k_bcycle_start(BatchKrylov K, cudaGraphConditionalHandle inner, int use_cond) {
    __shared__ int anyrun;
    if (threadIdx.x == 0) anyrun = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < K.npair; p += blockDim.x) {
        double *g = K.g + (int64_t)p * (K.m + 2);
        for (int i = 0; i <= K.m; ++i) g[i] = 0.0;
        g[0] = sqrt(K.rn2[p]);
        K.run[p] = K.active[p];
        K.jdone[p] = 0;
        if (K.active[p]) anyrun = 1;
    }
    __syncthreads();
    sys_flags(K);
    if (threadIdx.x == 0) {
        *K.j = 0;
        K.any[0] = anyrun;
        if (use_cond) cudaGraphSetConditional(inner, anyrun ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(256)
k_bscale(const BatchSegs S, BatchKrylov K, const double *__restrict__ r, double *__restrict__ V,
         double *__restrict__ vin) {
    const int c = blockIdx.x, s = S.cta_sys[c];
    __shared__ double inv[R8];
    if (threadIdx.x < R8) {
        const int p = s * R8 + threadIdx.x;
        inv[threadIdx.x] = K.active[p] ? 1.0 / sqrt(K.rn2[p]) : 0.0;
    }
    __syncthreads();
    for (int64_t idx = S.cta_r0[c] * R8 + threadIdx.x; idx < S.cta_r1[c] * R8; idx += blockDim.x) {
        const double v = r[idx] * inv[idx % R8];
        V[idx] = v;
        vin[idx] = v;
    }
}

// End of a step: next column while any pair is still running.
__global__ void k_bstep_end(BatchKrylov K, cudaGraphConditionalHandle inner, int use_cond) {
    __shared__ int anyrun;
    if (threadIdx.x == 0) anyrun = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < K.npair; p += blockDim.x)
        if (K.run[p]) anyrun = 1;
    sys_flags(K);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (anyrun) *K.j += 1;
        K.any[0] = anyrun;
        if (use_cond) cudaGraphSetConditional(inner, anyrun ? 1u : 0u);
    }
}

// y_p = R_p^{-1} g_p (one thread per pair).
__global__ void k_blsq(BatchKrylov K) {
    const int m = K.m, m1 = m + 1;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < K.npair; p += gridDim.x * blockDim.x) {
        const int jd = K.active[p] ? K.jdone[p] : 0;
        const double *H = K.H + (int64_t)p * m1 * m;
        const double *g = K.g + (int64_t)p * (m + 2);
        double *y = K.y + (int64_t)p * (m + 2);
        for (int i = jd - 1; i >= 0; --i) {
            double sum = g[i];
            for (int t = i + 1; t < jd; ++t) sum -= H[(int64_t)t * m1 + i] * y[t];
            y[i] = sum / H[(int64_t)i * m1 + i];
        }
        for (int i = jd; i <= m; ++i) y[i] = 0.0;
    }
}

// x_p += Z_p y_p
__global__ void __launch_bounds__(256)
k_bupdate_x(const BatchSegs S, BatchKrylov K, const double *__restrict__ Z, int64_t ldz, double *__restrict__ x) {
    __shared__ double ys[R8][kMaxCols + 1];      // odd row stride: the 8 rhs of a warp in 8 banks
    __shared__ int jd[R8];
    const int c = blockIdx.x, s = S.cta_sys[c];
    if (threadIdx.x < R8) {
        const int p = s * R8 + threadIdx.x;
        jd[threadIdx.x] = K.active[p] ? K.jdone[p] : 0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < R8 * K.m; idx += blockDim.x) {
        const int rr = idx / K.m, cc = idx % K.m;
        ys[rr][cc] = K.y[(int64_t)(s * R8 + rr) * (K.m + 2) + cc];
    }
    __syncthreads();
    for (int64_t idx = S.cta_r0[c] * R8 + threadIdx.x; idx < S.cta_r1[c] * R8; idx += blockDim.x) {
        const int rr = (int)(idx % R8);
        double acc = x[idx];
        for (int cc = 0; cc < jd[rr]; ++cc) acc += Z[(int64_t)cc * ldz + idx] * ys[rr][cc];
        x[idx] = acc;
    }
}

// End of a cycle: true residual test per pair (rn2 holds ||b - A x||^2).
__global__ void k_bcycle_end(BatchKrylov K, cudaGraphConditionalHandle outer, int use_cond) {
    __shared__ int anyact, jmax;
    if (threadIdx.x == 0) { anyact = 0; jmax = 0; }
    __syncthreads();
    for (int p = threadIdx.x; p < K.npair; p += blockDim.x) {
        if (!K.active[p]) continue;
        atomicMax(&jmax, K.jdone[p]);
        K.its[p] += K.jdone[p];
        const double rn = sqrt(K.rn2[p]);
        if (!isfinite(rn) || K.bad[p]) {
            K.bad[p] = 1;
            K.active[p] = 0;
        } else if (rn <= K.tol[p]) {
            K.conv[p] = 1;
            K.active[p] = 0;
        } else {
            K.restarts[p] += 1;
            anyact = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *K.iters += jmax;
        const int again = anyact && *K.iters < *K.maxit;
        K.any[1] = again;
        if (use_cond) cudaGraphSetConditional(outer, again ? 1u : 0u);
    }
}

// Gather / scatter between the user layout (system s: n_s x nrhs, column-major)
// and the batch layout (permuted rows, 8 interleaved rhs).
__global__ void k_bgather(int64_t nrows, const int32_t *__restrict__ sys_of, const int64_t *__restrict__ perm_g,
                          const int64_t *__restrict__ usr_off, const int64_t *__restrict__ nsz, int nrhs,
                          const double *__restrict__ src, double *__restrict__ dst) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * R8) return;
    const int64_t g = idx / R8;
    const int r = (int)(idx % R8);
    const int s = sys_of[g];
    dst[idx] = r < nrhs ? src[usr_off[s] + (int64_t)r * nsz[s] + perm_g[g]] : 0.0;
}
__global__ void k_bscatter(int64_t nrows, const int32_t *__restrict__ sys_of, const int64_t *__restrict__ perm_g,
                           const int64_t *__restrict__ usr_off, const int64_t *__restrict__ nsz, int nrhs,
                           const double *__restrict__ src, double *__restrict__ dst) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * R8) return;
    const int64_t g = idx / R8;
    const int r = (int)(idx % R8);
    if (r >= nrhs) return;
    const int s = sys_of[g];
    dst[usr_off[s] + (int64_t)r * nsz[s] + perm_g[g]] = src[idx];
}

// ---- launchers ----------------------------------------------------------------------------
template <int MODE, int RPC>
static void launch_btrsv_smem(const BatchLevel &lv, size_t smem_bytes, const double *in, float *work,
                              double *out_final, float *scratch, cudaStream_t st) {
    k_btrsv<MODE, true, RPC><<<lv.nblk * (R8 / RPC), kBatchTrsvThreads, smem_bytes, st>>>(lv, in, work, out_final,
                                                                                         scratch);
}
template <int MODE>
static void launch_btrsv_mode(const BatchLevel &lv, int rpc, size_t smem_bytes, const double *in, float *work,
                              double *out_final, float *scratch, cudaStream_t st) {
    switch (rpc) {
        case 8: launch_btrsv_smem<MODE, 8>(lv, smem_bytes, in, work, out_final, scratch, st); break;
        case 4: launch_btrsv_smem<MODE, 4>(lv, smem_bytes, in, work, out_final, scratch, st); break;
        case 2: launch_btrsv_smem<MODE, 2>(lv, smem_bytes, in, work, out_final, scratch, st); break;
        case 1: launch_btrsv_smem<MODE, 1>(lv, smem_bytes, in, work, out_final, scratch, st); break;
        default:
            k_btrsv<MODE, false, R8><<<lv.nblk, kBatchTrsvThreads, kRingBytes, st>>>(lv, in, work, out_final, scratch);
    }
}
// rpc: right-hand sides per CTA (8, 4, 2, 1: vector in shared memory of
// kRingBytes + rows * rpc * 4 bytes), 0: vector in global memory
void launch_btrsv(const BatchLevel &lv, int mode, int rpc, size_t smem_bytes, const double *in, float *work,
                  double *out_final, float *scratch, cudaStream_t st) {
    if (lv.nblk == 0) return;
    if (mode == 0) launch_btrsv_mode<0>(lv, rpc, smem_bytes, in, work, out_final, scratch, st);
    else launch_btrsv_mode<1>(lv, rpc, smem_bytes, in, work, out_final, scratch, st);
    count_launch();
}
template <int RPC>
static void set_btrsv_attr(int bytes) {
    cudaFuncSetAttribute(k_btrsv<0, true, RPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_btrsv<1, true, RPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
void set_btrsv_smem_limit(int bytes) {
    set_btrsv_attr<8>(bytes);
    set_btrsv_attr<4>(bytes);
    set_btrsv_attr<2>(bytes);
    set_btrsv_attr<1>(bytes);
    cudaFuncSetAttribute(k_btrsv<0, false, R8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
    cudaFuncSetAttribute(k_btrsv<1, false, R8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
}
void launch_bcouple(const BatchLevel &lv, const double *in, float *work, cudaStream_t st) {
    if (lv.ncta == 0) return;
    k_bcouple<<<lv.ncta, kBatchThreads, 0, st>>>(lv, in, work);
    count_launch();
}
void launch_blowrank(const BatchLevel &lv, float *work, cudaStream_t st) {
    if (lv.ncta == 0) return;
    k_blowrank<<<lv.ncta, kBatchThreads, 0, st>>>(lv, work);
    count_launch();
}
void launch_bspmv(int64_t nrows, const int64_t *rp, const int32_t *ci, const double *v, const double *x,
                  const double *b, double *y, double *zcol, const int32_t *jp, int64_t ld, cudaStream_t st,
                  const int32_t *sys_of, const int32_t *live) {
    const int64_t n = nrows * R8;
    if (n == 0) return;
    k_bspmv<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nrows, rp, ci, v, x, b, y, zcol, jp, ld, sys_of, live);
    count_launch();
}
void launch_bgs(int pass, const BatchSegs &S, const BatchKrylov &K, double *V, int64_t ldv, double *w,
                cudaStream_t st) {
    const size_t bytes = sizeof(double) * std::max(R8 * (K.m + 1), kGs1Threads);
    if (pass == 1) {
        k_bgs_dots<1><<<S.ncta, kGs1Threads, bytes, st>>>(S, K, V, ldv, w);
    } else {
        k_bgs_sub<<<S.ncta, 256, 0, st>>>(S, K, V, ldv, w);
        count_launch();
        k_bgs_dots<2><<<S.ncta, kGs1Threads, bytes, st>>>(S, K, V, ldv, w);
    }
    count_launch();
}
void launch_bgs_subnorm(const BatchSegs &S, const BatchKrylov &K, double *V, int64_t ldv, double *w,
                        cudaStream_t st) {
    k_bgs_subnorm<<<S.ncta, 256, 0, st>>>(S, K, V, ldv, w);
    count_launch();
}
void launch_bgs_final(const BatchSegs &S, const BatchKrylov &K, double *V, int64_t ldv, const double *w, double *vin,
                      cudaStream_t st) {
    k_bgs_final<<<S.ncta, 256, 0, st>>>(S, K, V, ldv, w, vin);
    count_launch();
}
void launch_bnorm2(const BatchSegs &S, double *partial, const double *x, double *out, cudaStream_t st) {
    k_bnorm2<<<S.ncta, 256, 0, st>>>(S, partial, x, out);
    count_launch();
}
void launch_binit(const BatchKrylov &K, double rtol, int maxit, cudaStream_t st) {
    k_binit<<<(K.npair + 255) / 256, 256, 0, st>>>(K, rtol, maxit);
    count_launch();
}
void launch_bcycle_start(const BatchKrylov &K, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
    k_bcycle_start<<<1, 1024, 0, st>>>(K, h, use_cond);
    count_launch();
}
void launch_bscale(const BatchSegs &S, const BatchKrylov &K, const double *r, double *V, double *vin, cudaStream_t st) {
    k_bscale<<<S.ncta, 256, 0, st>>>(S, K, r, V, vin);
    count_launch();
}
void launch_bstep_end(const BatchKrylov &K, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
    k_bstep_end<<<1, 1024, 0, st>>>(K, h, use_cond);
    count_launch();
}
void launch_blsq(const BatchKrylov &K, cudaStream_t st) {
    k_blsq<<<(K.npair + 127) / 128, 128, 0, st>>>(K);
    count_launch();
}
void launch_bupdate_x(const BatchSegs &S, const BatchKrylov &K, const double *Z, int64_t ldz, double *x,
                      cudaStream_t st) {
    k_bupdate_x<<<S.ncta, 256, 0, st>>>(S, K, Z, ldz, x);
    count_launch();
}
void launch_bcycle_end(const BatchKrylov &K, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
    k_bcycle_end<<<1, 1024, 0, st>>>(K, h, use_cond);
    count_launch();
}
void launch_bgather(int64_t nrows, const int32_t *sys_of, const int64_t *perm_g, const int64_t *usr_off,
                    const int64_t *nsz, int nrhs, const double *src, double *dst, cudaStream_t st) {
    const int64_t n = nrows * R8;
    if (n == 0) return;
    k_bgather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nrows, sys_of, perm_g, usr_off, nsz, nrhs, src, dst);
    count_launch();
}
void launch_bscatter(int64_t nrows, const int32_t *sys_of, const int64_t *perm_g, const int64_t *usr_off,
                     const int64_t *nsz, int nrhs, const double *src, double *dst, cudaStream_t st) {
    const int64_t n = nrows * R8;
    if (n == 0) return;
    k_bscatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nrows, sys_of, perm_g, usr_off, nsz, nrhs, src, dst);
    count_launch();
}

}  // namespace gemslr
