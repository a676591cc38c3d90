// Device primitives shared by the kernels: warp reductions, deterministic
// column reductions of per-CTA partial sums, the mbarrier / bulk-copy (TMA,
// non-tensor) PTX of the staged substitution kernels, and the lane-per-row
// chunk consumer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace gemslr {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// Column sums of per-CTA partials [nparts][ncols1] into out[0..ncols1) (shared
// memory), by all warps of the finishing CTA: warp w owns columns w, w+nw, ...,
// its lanes stride over the partials (callers use 256-thread CTAs: 8 warps),
// so every lane keeps up to kColsPerWarp
// independent loads in flight; the summation order is fixed (deterministic).
constexpr int kColsPerWarp = (kMaxCols + 1 + 7) / 8;
template <typename T>
__device__ void reduce_columns(const T *partial, int nparts, int ncols1, T *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T acc[kColsPerWarp];
#pragma unroll
    for (int u = 0; u < kColsPerWarp; ++u) acc[u] = 0;
    for (int p = lane; p < nparts; p += 32) {
        const T *row = partial + (int64_t)p * ncols1;
#pragma unroll
        for (int u = 0; u < kColsPerWarp; ++u) {
            const int c = warp + nw * u;
            if (c < ncols1) acc[u] += __ldcg(row + c);
        }
    }
#pragma unroll
    for (int u = 0; u < kColsPerWarp; ++u) {
        const int c = warp + nw * u;          // uniform over the warp
        if (c < ncols1) {
            const T v = warp_sum(acc[u]);
            if (lane == 0) out[c] = v;
        }
    }
    __syncthreads();
}

// ---- mbarrier / bulk-copy primitives (sm_90+ PTX) ------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Polling wait (no suspension) for the consumers' critical path, bounded like wait_bounded.
__device__ __forceinline__ bool poll_bounded(uint64_t *bar, unsigned parity, volatile int *abort_flag) {
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned spins = 0;
    while (!mbar_test_wait(bar, parity)) {
        if ((++spins & 63u) == 0u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > 4000000000ll) return false;
        }
    }
    return true;
}
__device__ __forceinline__ void consumer_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsumerWarps) : "memory");
}
// One bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Every wait is bounded: about 2 s of clock cycles, or until another warp of
// the CTA has raised `abort`.
constexpr long long kSpinCycles = 4000000000ll;

__device__ __forceinline__ bool wait_bounded(uint64_t *bar, unsigned parity, volatile int *abort_flag) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (abort_flag && *abort_flag) return false;
        if (clock64() - t0 > kSpinCycles) return false;
    }
    return true;
}

// Registers holding one row slot of a chunk (lane-per-row layout).
constexpr int kRegEntries = 16;
template <typename VT>
struct RowRegs {
    int row, len, nrow, S, st;
    int col[kRegEntries];
    VT val[kRegEntries];
    VT dinv;
    bool upper, active;
};

// Wait for chunk k and copy this lane's row slot into registers.
template <typename VT>
__device__ __forceinline__ bool fetch_row(const unsigned char *ring, uint64_t *full, volatile int *abort_flag,
                                          int k, int lane, RowRegs<VT> &R) {
    const int st = k % kStages;
    R.st = st;
    if (!poll_bounded(&full[st], (k / kStages) & 1, abort_flag)) return false;
    const int *hdr = reinterpret_cast<const int *>(ring + (size_t)st * kStageBytes);
    R.nrow = hdr[0];
    R.S = hdr[1];
    R.upper = hdr[2] != 0;
    const int pr = (R.nrow + 3) & ~3;
    const int *rows = hdr + 4;
    const int *lens = rows + pr;
    const int *cols = lens + pr;
    const int ne = R.S * R.nrow;
    const VT *vals = reinterpret_cast<const VT *>(cols + ((ne + 3) & ~3));
    const int nv = (int)((((size_t)ne * sizeof(VT) + 15) & ~(size_t)15) / sizeof(VT));
    R.active = lane < R.nrow;
    R.row = R.active ? rows[lane] : 0;
    R.len = R.active ? lens[lane] : 0;
    R.dinv = (R.active && R.upper) ? vals[nv + lane] : (VT)1;
#pragma unroll
    for (int q = 0; q < kRegEntries; ++q) {
        if (q < R.len) {
            R.col[q] = cols[q * R.nrow + lane];
            R.val[q] = vals[q * R.nrow + lane];
        } else {
            R.col[q] = 0;
            R.val[q] = 0;
        }
    }
    return true;
}

// Named barriers 2 .. 1+kConsumerWarps hand the sweep from one consumer warp
// to the next (64 threads: the signalling warp arrives, the next one waits).
__device__ __forceinline__ void handoff_wait(int warp) {
    asm volatile("bar.sync %0, 64;" ::"r"(2 + warp) : "memory");
}
__device__ __forceinline__ void handoff_signal(int next_warp) {
    asm volatile("bar.arrive %0, 64;" ::"r"(2 + next_warp) : "memory");
}

// Lane-per-row substitutions (FP32).  Chunk k belongs to consumer warp
// k % kConsumerWarps.  A warp loads its next chunk's rows, columns and values
// into registers while the other warps work, then waits for the previous
// chunk's warp, gathers x, computes its rows, stores them and hands on; the
// barrier orders the stores before the next warp's gathers.  Every warp runs
// the same sequence of waits and signals whatever happens (an expired wait
// only skips the arithmetic), so the hand-off chain always completes.
template <typename VT>
__device__ void consume_chunks_round_robin(const unsigned char *ring, uint64_t *full, uint64_t *empty,
                                           volatile int *abort_flag, int nchunk, VT *xs, int warp, int lane) {
    constexpr int NW = kConsumerWarps;
    bool ok = true;
    for (int k = warp; k < nchunk; k += NW) {
        RowRegs<VT> R;
        if (ok) ok = fetch_row<VT>(ring, full, abort_flag, k, lane, R);
        if (!ok && lane == 0) *abort_flag = 1;
        if (k > 0) handoff_wait(warp);
        if (ok && !*abort_flag) {
            VT xv[kRegEntries];
#pragma unroll
            for (int q = 0; q < kRegEntries; ++q) xv[q] = (q < R.len) ? xs[R.col[q]] : (VT)0;
            const VT self = R.active ? xs[R.row] : (VT)0;
            VT a0 = 0, a1 = 0;
#pragma unroll
            for (int q = 0; q < kRegEntries; q += 2) {
                a0 += R.val[q] * xv[q];
                a1 += R.val[q + 1] * xv[q + 1];
            }
            if (R.len > kRegEntries) {          // long rows: the rest straight from the staged chunk
                const int *hdr = reinterpret_cast<const int *>(ring + (size_t)R.st * kStageBytes);
                const int pr = (R.nrow + 3) & ~3;
                const int *cols = hdr + 4 + 2 * pr;
                const int ne = R.S * R.nrow;
                const VT *vals = reinterpret_cast<const VT *>(cols + ((ne + 3) & ~3));
                for (int q = kRegEntries; q < R.len; ++q) a0 += vals[q * R.nrow + lane] * xs[cols[q * R.nrow + lane]];
            }
            if (R.active) xs[R.row] = (self - (a0 + a1)) * R.dinv;
        }
        __syncwarp();
        if (k + 1 < nchunk) handoff_signal((warp + 1) % NW);
        if (ok && lane == 0) mbar_arrive(&empty[R.st]);
    }
}

}  // namespace
}  // namespace gemslr
