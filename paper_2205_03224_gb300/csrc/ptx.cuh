// Device primitives shared by the kernels: warp reductions, deterministic
// column reductions of per-CTA partial sums, the mbarrier / bulk-copy (TMA,
// non-tensor) PTX of the staged substitution kernels, and the lane-per-row
// chunk consumer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "zcomplex.cuh"

namespace gemslr {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}


// Column sums of per-CTA partials (column-major: partial c of CTA p at
// c * nparts + p, so a warp's loads of one column are contiguous) into
// out[0..ncols1) (shared memory), by all warps of the finishing CTA.  Warp w
// takes columns w, w+nw, w+2nw, w+3nw together; its lanes load up to eight
// partials each for all four columns before any addition (one memory round
// trip per pass of 256 CTAs), add them in a fixed pairwise tree and finish
// with a warp reduction.  The summation order is fixed (deterministic).  Short dependent
// chains matter here: one FP64 add takes on the order of a hundred cycles on
// this part when nothing else is in flight.
template <typename T>
__device__ void reduce_columns(const T *partial, int nparts, int ncols1, T *out) {
    constexpr int RP = 8, CW = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int cb = warp; cb < ncols1; cb += CW * nw) {
        T acc[CW];
#pragma unroll
        for (int u = 0; u < CW; ++u) acc[u] = 0;
        for (int p0 = 0; p0 < nparts; p0 += 32 * RP) {
            T v[CW][RP];
#pragma unroll
            for (int u = 0; u < CW; ++u) {
                const int c = cb + u * nw;
#pragma unroll
                for (int q = 0; q < RP; ++q) {
                    const int p = p0 + q * 32 + lane;
                    v[u][q] = (c < ncols1 && p < nparts) ? ldcg(partial + (int64_t)c * nparts + p) : (T)0;
                }
            }
#pragma unroll
            for (int u = 0; u < CW; ++u)
                acc[u] += ((v[u][0] + v[u][1]) + (v[u][2] + v[u][3])) + ((v[u][4] + v[u][5]) + (v[u][6] + v[u][7]));
        }
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            const int c = cb + u * nw;          // uniform over the warp
            if (c < ncols1) {
                const T t = warp_sum(acc[u]);
                if (lane == 0) out[c] = t;
            }
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
// Every wait is bounded: about 2 s of clock cycles (or `limit`), or until
// another warp of the CTA has raised `abort`.
constexpr long long kSpinCycles = 4000000000ll;

// Polling wait (no suspension) for the consumers' critical path, bounded like wait_bounded.
__device__ __forceinline__ bool poll_bounded(uint64_t *bar, unsigned parity, volatile int *abort_flag,
                                             long long limit = kSpinCycles) {
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned spins = 0;
    while (!mbar_test_wait(bar, parity)) {
        if ((++spins & 63u) == 0u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) return false;
        }
    }
    return true;
}
__device__ __forceinline__ void consumer_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsumerWarps) : "memory");
}
// One bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16).  The factor chunks are read once per application, so the copy marks
// them evict-first in L2: the vectors that the substitutions gather from (in
// global memory for blocks too large for shared memory) keep their L2 lines.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ bool wait_bounded(uint64_t *bar, unsigned parity, volatile int *abort_flag,
                                             long long limit = kSpinCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (abort_flag && *abort_flag) return false;
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// Producer warp of the staged substitutions: streams the chunks [c0, c1)
// (byte ranges off[c] .. off[c+1] of data) into the ring, CPG chunks per
// bulk copy: group g goes to slot g % kGroups and completes on
// full[slot]; a slot is reused once its consumers have arrived on
// empty[slot].  The group offsets are read 32 groups at a time by the whole
// warp (the next batch while the current one is issued), so that no copy
// waits on a global load of its own size; lane 0 issues the copies.  On an
// expired wait the CTA's abort flag and the device error word are set.
// Before returning, lane 0 waits for the copies still in flight.
template <int CPG, int SB = kStageBytes>
__device__ __forceinline__ void produce_chunks(const unsigned char *data, const int64_t *off, int c0, int c1,
                                               unsigned char *ring, uint64_t *full, uint64_t *empty,
                                               volatile int *abort_flag, int32_t *err, int lane) {
    constexpr int kGroups = kRingData / (CPG * SB), kGroupBytes = CPG * SB;
    const int ngroup = (c1 - c0 + CPG - 1) / CPG;
    auto group_range = [&](int g, int64_t &a, int64_t &b) {
        a = off[c0 + CPG * g];
        b = off[min(c0 + CPG * (g + 1), c1)];
    };
    int issued = 0;
    int64_t o0 = 0, o1 = 0;
    if (lane < ngroup) group_range(lane, o0, o1);
    for (int base = 0; base < ngroup; base += 32) {
        int64_t n0 = 0, n1 = 0;
        if (base + 32 + lane < ngroup) group_range(base + 32 + lane, n0, n1);
        const int cnt = min(32, ngroup - base);
        bool ok = true;
        for (int t = 0; t < cnt; ++t) {
            const int64_t s0 = __shfl_sync(0xffffffffu, o0, t), s1 = __shfl_sync(0xffffffffu, o1, t);
            const int g = base + t, slot = g % kGroups;
            if (g >= kGroups) {
                const bool got = lane == 0 ? wait_bounded(&empty[slot], ((g / kGroups) - 1) & 1, abort_flag) : true;
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) {
                        *abort_flag = 1;
                        atomicExch(err, 1);
                    }
                    ok = false;
                    break;
                }
            }
            if (lane == 0) {
                const unsigned bytes = (unsigned)(s1 - s0);
                mbar_expect_tx(&full[slot], bytes);
                bulk_load(ring + (size_t)slot * kGroupBytes, data + s0, bytes, &full[slot]);
            }
            issued = g + 1;
        }
        if (!ok) break;
        o0 = n0;
        o1 = n1;
    }
    if (lane == 0)
        for (int g = issued > kGroups ? issued - kGroups : 0; g < issued; ++g)
            wait_bounded(&full[g % kGroups], (g / kGroups) & 1, nullptr);
}

// Bytes of one slice, and of one chunk (a slice and, while their headers say
// so, the slices after it); see kernels.cuh.
template <typename VT>
__device__ __forceinline__ int slice_size(const int *hdr) {
    const int nrow = hdr[0], S = hdr[1], pr = (nrow + 3) & ~3, ne = S * nrow;
    return 16 + 8 * pr + ((ne * 4 + 15) & ~15) + ((ne * (int)sizeof(VT) + 15) & ~15) +
           (hdr[2] ? ((nrow * (int)sizeof(VT) + 15) & ~15) : 0);
}
template <typename VT>
__device__ __forceinline__ int chunk_size(const int *hdr) {
    int a = 0;
    for (int t = 0; t < kMaxSlices; ++t) {
        const int *h = hdr + a / 4;
        a += slice_size<VT>(h);
        if (!h[3]) break;
    }
    return a;
}

// Wait until chunk k (block-relative) is in shared memory and return it: its
// group of CPG chunks is in slot (k / CPG) % kGroups, after the chunks
// before it.
template <typename VT, int CPG, int SB = kStageBytes>
__device__ __forceinline__ const unsigned char *wait_chunk(const unsigned char *ring, uint64_t *full,
                                                           volatile int *abort_flag, int k) {
    constexpr int kGroups = kRingData / (CPG * SB), kGroupBytes = CPG * SB;
    const int g = k / CPG, slot = g % kGroups;
    if (!poll_bounded(&full[slot], (g / kGroups) & 1, abort_flag)) return nullptr;
    const unsigned char *p = ring + (size_t)slot * kGroupBytes;
    for (int i = 0; i < k % CPG; ++i) p += chunk_size<VT>(reinterpret_cast<const int *>(p));
    return p;
}

// For consumers that take the chunks in order: chunk k follows chunk k-1
// (at prev) in the same group, else it starts a group that must be waited for.
template <typename VT, int CPG, int SB = kStageBytes>
__device__ __forceinline__ const unsigned char *next_chunk(const unsigned char *ring, uint64_t *full,
                                                           volatile int *abort_flag, int k,
                                                           const unsigned char *prev) {
    constexpr int kGroups = kRingData / (CPG * SB), kGroupBytes = CPG * SB;
    if (k % CPG != 0) return prev + chunk_size<VT>(reinterpret_cast<const int *>(prev));
    const int g = k / CPG, slot = g % kGroups;
    if (!poll_bounded(&full[slot], (g / kGroups) & 1, abort_flag)) return nullptr;
    return ring + (size_t)slot * kGroupBytes;
}

// Ring slot of chunk k for CPG chunks of at most SB bytes per copy.
template <int CPG, int SB = kStageBytes>
__device__ __forceinline__ int chunk_slot(int k) { return (k / CPG) % (kRingData / (CPG * SB)); }

// Registers holding one row slot of a chunk (lane-per-row layout): NE entry
// slots (the launch picks NE >= the level's longest row where it can; longer
// rows finish from shared memory).
constexpr int kRegEntries = 16;
template <typename VT, int NE = kRegEntries>
struct RowRegs {
    const unsigned char *base;
    int row, len, nrow, S;
    int col[NE];               // byte offsets into x (column * sizeof(VT)), computed before the wait
    VT val[NE];
    VT dinv;
    bool upper, active;
};

// Copy this lane's row slot of the chunk at p (shared memory) into registers.
// Branch-free: every lane loads all kRegEntries slots, at indices clamped into
// the chunk (inactive lanes read the last row slot, slots past S read slot
// S-1), and keeps zeros (column 0, value 0) past its row's length, so that all
// the loads of a chunk are in flight together.
template <typename VT, int NE>
__device__ __forceinline__ void fetch_row(const unsigned char *p, int lane, RowRegs<VT, NE> &R) {
    const int *hdr = reinterpret_cast<const int *>(p);
    R.base = p;
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
    const int t = R.active ? lane : R.nrow - 1;
    const int row = rows[t], len = lens[t];
    R.row = row;
    R.len = R.active ? len : 0;
    const VT di = vals[R.upper ? nv + t : 0];       // L chunks have no 1/u_ii (and >= 1 entry)
    R.dinv = (R.active && R.upper) ? di : (VT)1;
    const int smax = R.S > 0 ? R.S - 1 : 0;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        const int e = min(q, smax) * R.nrow + t;
        const int c = cols[e];
        const VT v = vals[e];
        const bool live = q < R.len;
        R.col[q] = live ? c * (int)sizeof(VT) : 0;
        R.val[q] = live ? v : (VT)0;
    }
}

// x_row = x_row * dinv + sum_q val_q x_col_q for this lane's row slot (the
// values are stored negated and, in U chunks, divided by u_row,row).
template <typename VT, int NE>
__device__ __forceinline__ void solve_row(const RowRegs<VT, NE> &R, VT *xs, int lane) {
    static_assert(NE % 2 == 0, "two partial sums");
    VT xv[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q)            // padded slots: x_0 * 0
        xv[q] = *reinterpret_cast<const VT *>(reinterpret_cast<const unsigned char *>(xs) + R.col[q]);
    const VT self = xs[R.row];                 // loaded with the gathers, used after the chains
    VT a0 = 0, a1 = 0;
#pragma unroll
    for (int q = 0; q < NE; q += 2) {
        a0 += R.val[q] * xv[q];
        a1 += R.val[q + 1] * xv[q + 1];
    }
    if (R.len > NE) {                   // long rows: the rest straight from the staged slice
        const int pr = (R.nrow + 3) & ~3;
        const int *cols = reinterpret_cast<const int *>(R.base) + 4 + 2 * pr;
        const int ne = R.S * R.nrow;
        const VT *vals = reinterpret_cast<const VT *>(cols + ((ne + 3) & ~3));
        for (int q = NE; q < R.len; ++q) a0 += vals[q * R.nrow + lane] * xs[cols[q * R.nrow + lane]];
    }
    if (R.active) xs[R.row] = fmaf(self, R.dinv, a0 + a1);
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
// k % kConsumerWarps (one chunk of every group).  A warp loads its next
// chunk (one to kMaxSlices slices: consecutive wavefronts) into registers
// while the other warps work, then waits for the previous chunk's warp,
// gathers x, computes its rows (each later slice after a __syncwarp), stores
// them and hands on; the barrier orders the stores before the next warp's
// gathers.  Every warp runs the same sequence of waits and signals whatever
// happens (an expired wait only skips the arithmetic), so the hand-off chain
// always completes.
template <typename VT, int NE, int SB>
__device__ void consume_chunks_round_robin(const unsigned char *ring, uint64_t *full, uint64_t *empty,
                                           volatile int *abort_flag, int nchunk, VT *xs, int warp, int lane) {
    static_assert(kConsumerWarps == kGroupChunks, "one chunk of every group per consumer warp");
    static_assert(kMaxSlices == 4, "four slice registers");
    constexpr int NW = kConsumerWarps;
    bool ok = true;
    for (int k = warp; k < nchunk; k += NW) {
        RowRegs<VT, NE> R0, R1, R2, R3;
        const unsigned char *p = ok ? wait_chunk<VT, kGroupChunks, SB>(ring, full, abort_flag, k) : nullptr;
        ok = p != nullptr;
        if (!ok && lane == 0) *abort_flag = 1;
        int ns = 0;                             // slices of the chunk (uniform over the warp)
        if (ok) {
            const unsigned char *q = p;
            fetch_row<VT, NE>(q, lane, R0);
            ns = 1;
            if (reinterpret_cast<const int *>(q)[3]) {
                q += slice_size<VT>(reinterpret_cast<const int *>(q));
                fetch_row<VT, NE>(q, lane, R1);
                ns = 2;
                if (reinterpret_cast<const int *>(q)[3]) {
                    q += slice_size<VT>(reinterpret_cast<const int *>(q));
                    fetch_row<VT, NE>(q, lane, R2);
                    ns = 3;
                    if (reinterpret_cast<const int *>(q)[3]) {
                        q += slice_size<VT>(reinterpret_cast<const int *>(q));
                        fetch_row<VT, NE>(q, lane, R3);
                        ns = 4;
                    }
                }
            }
        }
        const bool go = ok && !*abort_flag;     // read before the wait, off the critical path
        if (k > 0) handoff_wait(warp);
        if (go) {
            // each slice's rows are stored before the next slice's gathers
            solve_row<VT, NE>(R0, xs, lane);
            if (ns > 1) {
                __syncwarp();
                solve_row<VT, NE>(R1, xs, lane);
            }
            if (ns > 2) {
                __syncwarp();
                solve_row<VT, NE>(R2, xs, lane);
            }
            if (ns > 3) {
                __syncwarp();
                solve_row<VT, NE>(R3, xs, lane);
            }
        }
        // bar.arrive orders each lane's own stores before the next warp's gathers
        if (k + 1 < nchunk) handoff_signal((warp + 1) % NW);
        __syncwarp();                           // every lane is done with the staged chunk
        if (ok && lane == 0) mbar_arrive(&empty[chunk_slot<kGroupChunks, SB>(k)]);
    }
}

}  // namespace
}  // namespace gemslr
