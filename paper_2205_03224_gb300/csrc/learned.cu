// Learned interface correction: network kernels (forward, backward, Adam),
// training-data generation and the in-apply stage.  See learned.cuh.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "device.h"
#include "learned.cuh"
#include "ptx.cuh"

namespace gemslr {

namespace {

constexpr int kConvSitesPerCta = 32;      // 8 thread rows x 4 sites each
constexpr int kMaxCh = 32;

// y[n, s, co] = b[co] + sum_t sum_ci W[t, ci, co] x[n, nbr[s, t], ci]; z = y, h = relu(y) (if relu).
// Block (32 co, 8 rows); every thread keeps 4 sites; W[t] staged in shared memory per tap.
__global__ void __launch_bounds__(256)
k_conv_fwd(int S, int Cin, int Cout, const float *__restrict__ x, const __nv_bfloat16 *__restrict__ W,
           const float *__restrict__ b, const int32_t *__restrict__ nbr, float *__restrict__ z, float *__restrict__ h,
           int relu) {
    __shared__ float Ws[kMaxCh * kMaxCh];
    const int co = threadIdx.x, ty = threadIdx.y;
    const int n = blockIdx.y;
    const int s0 = blockIdx.x * kConvSitesPerCta;
    float acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = (co < Cout) ? b[co] : 0.f;
    const float *xn = x + (int64_t)n * S * Cin;
    for (int t = 0; t < 27; ++t) {
        __syncthreads();
        for (int i = ty * 32 + co; i < Cin * Cout; i += 256) Ws[i] = __bfloat162float(W[(int64_t)t * Cin * Cout + i]);
        __syncthreads();
        if (co >= Cout) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = s0 + ty + 8 * j;
            if (s >= S) continue;
            const int src = nbr[s * 27 + t];
            if (src < 0) continue;
            const float *xr = xn + (int64_t)src * Cin;
            float a = 0.f;
            for (int ci = 0; ci < Cin; ++ci) a += Ws[ci * Cout + co] * xr[ci];
            acc[j] += a;
        }
    }
    if (co >= Cout) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int s = s0 + ty + 8 * j;
        if (s >= S) continue;
        const int64_t o = ((int64_t)n * S + s) * Cout + co;
        z[o] = acc[j];
        if (h) h[o] = relu ? fmaxf(acc[j], 0.f) : acc[j];
    }
}

// dx[n, u, ci] = sum_t sum_co W[t, ci, co] dy[n, nbr[u, 26 - t], co]
__global__ void __launch_bounds__(256)
k_conv_bwd_data(int S, int Cin, int Cout, const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ W,
                const int32_t *__restrict__ nbr, float *__restrict__ dx) {
    __shared__ float Wt[kMaxCh * kMaxCh];           // transposed: [co][ci]
    const int ci = threadIdx.x, ty = threadIdx.y;
    const int n = blockIdx.y;
    const int u0 = blockIdx.x * kConvSitesPerCta;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const float *dyn = dy + (int64_t)n * S * Cout;
    for (int t = 0; t < 27; ++t) {
        __syncthreads();
        for (int i = ty * 32 + ci; i < Cin * Cout; i += 256) {
            const int a = i / Cout, c = i % Cout;
            Wt[c * Cin + a] = __bfloat162float(W[(int64_t)t * Cin * Cout + i]);
        }
        __syncthreads();
        if (ci >= Cin) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int u = u0 + ty + 8 * j;
            if (u >= S) continue;
            const int s = nbr[u * 27 + (26 - t)];
            if (s < 0) continue;
            const float *g = dyn + (int64_t)s * Cout;
            float a = 0.f;
            for (int c = 0; c < Cout; ++c) a += Wt[c * Cin + ci] * g[c];
            acc[j] += a;
        }
    }
    if (ci >= Cin) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int u = u0 + ty + 8 * j;
        if (u < S) dx[((int64_t)n * S + u) * Cin + ci] = acc[j];
    }
}

// Per-chunk partial weight gradients: part[chunk][t][ci][co] = sum over the
// chunk's rows (n, s) of x[n, nbr[s, t], ci] dy[n, s, co].  Grid (27, nchunk).
__global__ void __launch_bounds__(256)
k_conv_bwd_w(int NS, int S, int Cin, int Cout, const float *__restrict__ x, const float *__restrict__ dy,
             const int32_t *__restrict__ nbr, int rows_per_chunk, float *__restrict__ part) {
    __shared__ float xs[32][kMaxCh + 1];
    __shared__ float gs[32][kMaxCh + 1];
    const int t = blockIdx.x, chunk = blockIdx.y;
    const int co = threadIdx.x, ty = threadIdx.y;          // ci = ty + 8*j
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int r0 = chunk * rows_per_chunk, r1 = min(NS, r0 + rows_per_chunk);
    for (int rb = r0; rb < r1; rb += 32) {
        __syncthreads();
        for (int i = ty * 32 + co; i < 32 * kMaxCh; i += 256) {
            const int rr = i / kMaxCh, c = i % kMaxCh;
            const int row = rb + rr;
            float xv = 0.f, gv = 0.f;
            if (row < r1) {
                const int n = row / S, s = row % S;
                const int src = nbr[s * 27 + t];
                if (c < Cin && src >= 0) xv = x[((int64_t)n * S + src) * Cin + c];
                if (c < Cout) gv = dy[(int64_t)row * Cout + c];
            }
            xs[rr][c] = xv;
            gs[rr][c] = gv;
        }
        __syncthreads();
        if (co < Cout) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ci = ty + 8 * j;
                if (ci >= Cin) continue;
                float a = 0.f;
                for (int rr = 0; rr < 32; ++rr) a += xs[rr][ci] * gs[rr][co];
                acc[j] += a;
            }
        }
    }
    if (co >= Cout) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int ci = ty + 8 * j;
        if (ci < Cin) part[(((int64_t)chunk * 27 + t) * Cin + ci) * Cout + co] = acc[j];
    }
}

// ---- tensor-core convolutions (BF16 mma.sync m16n8k16, FP32 accumulation) ----------------
// For the C -> C layers (C >= 8).  Every tap is a small GEMM over gathered
// rows: forward Y[s, co] += X[nbr(s, t), :] W_t, data gradient
// dX[u, ci] += dY[nbr(u, 26 - t), :] W_t^T, weight gradient
// dW_t[ci, co] += X[nbr(s, t), ci]^T dY[s, co].  The weights are BF16 as in
// the CUDA-core kernels; an FP32 activation or gradient operand is split into
// two BF16 terms (v = hi + lo, hi = bf16(v)), so that the products keep about
// 16 significant bits of it (weight gradients: hi*hi + hi*lo + lo*hi).
// Fragment coordinates of m16n8k16 (lane = 4 g + q):
//   A: a[0] (row g, cols 2q, 2q+1), a[1] (row g+8, same cols), a[2] (row g, cols 2q+8, 2q+9),
//      a[3] (row g+8, cols 2q+8, 2q+9); B: b[0] (rows 2q, 2q+1, col g), b[1] (rows 2q+8, 2q+9, col g);
//   D: d[0], d[1] (row g, cols 2q, 2q+1), d[2], d[3] (row g+8, same cols).
constexpr int kConvTcWarps = 4;                 // 16-site tiles per CTA (forward, data gradient)

__device__ __forceinline__ uint32_t bf16_pair(float lo_elem, float hi_elem) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t *>(&p);
}
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
    const float h0 = __bfloat162float(__float2bfloat16_rn(v0)), h1 = __bfloat162float(__float2bfloat16_rn(v1));
    hi = bf16_pair(h0, h1);
    lo = bf16_pair(v0 - h0, v1 - h1);
}
__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], const uint32_t b0, const uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// Two BF16 weights w[i0], w[i1] (element indices, out-of-range as zero) packed low/high.
__device__ __forceinline__ uint32_t w_pair(const __nv_bfloat16 *w, bool ok0, int i0, bool ok1, int i1) {
    const uint32_t lo = ok0 ? (uint32_t)__bfloat16_as_ushort(w[i0]) : 0u;
    const uint32_t hi = ok1 ? (uint32_t)__bfloat16_as_ushort(w[i1]) : 0u;
    return lo | (hi << 16);
}

// z = b + sum_t X[nbr(s, t)] W_t (h = relu(z) when relu); grid (ceil(S / 64), N),
// kConvTcWarps warps, dynamic shared memory 27 * Cin * Cout BF16 (all taps).
__global__ void __launch_bounds__(32 * kConvTcWarps)
k_conv_fwd_tc(int S, int Cin, int Cout, const float *__restrict__ x, const __nv_bfloat16 *__restrict__ W,
              const float *__restrict__ b, const int32_t *__restrict__ nbr, float *__restrict__ z,
              float *__restrict__ h, int relu) {
    extern __shared__ __align__(16) unsigned char conv_smem[];
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(conv_smem);
    const int nw = 27 * Cin * Cout;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) Ws[i] = W[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const int n = blockIdx.y;
    const int sa = (blockIdx.x * kConvTcWarps + warp) * 16 + g, sb = sa + 8;
    const float *xn = x + (int64_t)n * S * Cin;
    const int ntn = (Cout + 7) / 8;                  // n-tiles of 8 output channels (<= 4)
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c0 = nt * 8 + 2 * q;
        d[nt][0] = d[nt][2] = (c0 < Cout) ? b[c0] : 0.f;
        d[nt][1] = d[nt][3] = (c0 + 1 < Cout) ? b[c0 + 1] : 0.f;
    }
    for (int t = 0; t < 27; ++t) {
        const int src_a = sa < S ? nbr[sa * 27 + t] : -1, src_b = sb < S ? nbr[sb * 27 + t] : -1;
        for (int kk = 0; kk < Cin; kk += 16) {
            uint32_t ah[4], al[4];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {             // K columns 2q, 2q+1 (+8)
                const int ci = kk + 2 * q + 8 * hh;
                const float xa0 = (src_a >= 0 && ci < Cin) ? xn[(int64_t)src_a * Cin + ci] : 0.f;
                const float xa1 = (src_a >= 0 && ci + 1 < Cin) ? xn[(int64_t)src_a * Cin + ci + 1] : 0.f;
                const float xb0 = (src_b >= 0 && ci < Cin) ? xn[(int64_t)src_b * Cin + ci] : 0.f;
                const float xb1 = (src_b >= 0 && ci + 1 < Cin) ? xn[(int64_t)src_b * Cin + ci + 1] : 0.f;
                split2(xa0, xa1, ah[2 * hh], al[2 * hh]);
                split2(xb0, xb1, ah[2 * hh + 1], al[2 * hh + 1]);
            }
            const __nv_bfloat16 *wt = Ws + t * Cin * Cout;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                if (nt >= ntn) break;
                const int co = nt * 8 + g;
                const int r0 = kk + 2 * q, r1 = r0 + 8;   // K rows (input channels) of b[0], b[1]
                const bool okc = co < Cout;
                const uint32_t b0 = w_pair(wt, okc && r0 < Cin, r0 * Cout + co, okc && r0 + 1 < Cin, (r0 + 1) * Cout + co);
                const uint32_t b1 = w_pair(wt, okc && r1 < Cin, r1 * Cout + co, okc && r1 + 1 < Cin, (r1 + 1) * Cout + co);
                mma16816(d[nt], ah, b0, b1);
                mma16816(d[nt], al, b0, b1);
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        if (nt >= ntn) break;
        const int c0 = nt * 8 + 2 * q;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int s = e < 2 ? sa : sb, co = c0 + (e & 1);
            if (s < S && co < Cout) {
                const int64_t o = ((int64_t)n * S + s) * Cout + co;
                z[o] = d[nt][e];
                if (h) h[o] = relu ? fmaxf(d[nt][e], 0.f) : d[nt][e];
            }
        }
    }
}

// dx[n, u, ci] = sum_t sum_co W[t, ci, co] dy[n, nbr[u, 26 - t], co]; layout as k_conv_fwd_tc.
__global__ void __launch_bounds__(32 * kConvTcWarps)
k_conv_bwd_data_tc(int S, int Cin, int Cout, const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ W,
                   const int32_t *__restrict__ nbr, float *__restrict__ dx) {
    extern __shared__ __align__(16) unsigned char conv_smem[];
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(conv_smem);
    const int nw = 27 * Cin * Cout;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) Ws[i] = W[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const int n = blockIdx.y;
    const int ua = (blockIdx.x * kConvTcWarps + warp) * 16 + g, ub = ua + 8;
    const float *gn = dy + (int64_t)n * S * Cout;
    const int ntn = (Cin + 7) / 8;
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[nt][e] = 0.f;
    for (int t = 0; t < 27; ++t) {
        const int sa = ua < S ? nbr[ua * 27 + (26 - t)] : -1, sb = ub < S ? nbr[ub * 27 + (26 - t)] : -1;
        for (int kk = 0; kk < Cout; kk += 16) {
            uint32_t ah[4], al[4];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {             // K columns (output channels) 2q, 2q+1 (+8)
                const int co = kk + 2 * q + 8 * hh;
                const float ga0 = (sa >= 0 && co < Cout) ? gn[(int64_t)sa * Cout + co] : 0.f;
                const float ga1 = (sa >= 0 && co + 1 < Cout) ? gn[(int64_t)sa * Cout + co + 1] : 0.f;
                const float gb0 = (sb >= 0 && co < Cout) ? gn[(int64_t)sb * Cout + co] : 0.f;
                const float gb1 = (sb >= 0 && co + 1 < Cout) ? gn[(int64_t)sb * Cout + co + 1] : 0.f;
                split2(ga0, ga1, ah[2 * hh], al[2 * hh]);
                split2(gb0, gb1, ah[2 * hh + 1], al[2 * hh + 1]);
            }
            const __nv_bfloat16 *wt = Ws + t * Cin * Cout;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                if (nt >= ntn) break;
                const int ci = nt * 8 + g;                // B column (n) = input channel
                const int r0 = kk + 2 * q, r1 = r0 + 8;   // B rows (k) = output channels
                const bool okc = ci < Cin;
                const uint32_t b0 = w_pair(wt, okc && r0 < Cout, ci * Cout + r0, okc && r0 + 1 < Cout, ci * Cout + r0 + 1);
                const uint32_t b1 = w_pair(wt, okc && r1 < Cout, ci * Cout + r1, okc && r1 + 1 < Cout, ci * Cout + r1 + 1);
                mma16816(d[nt], ah, b0, b1);
                mma16816(d[nt], al, b0, b1);
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        if (nt >= ntn) break;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int u = e < 2 ? ua : ub, ci = nt * 8 + 2 * q + (e & 1);
            if (u < S && ci < Cin) dx[((int64_t)n * S + u) * Cin + ci] = d[nt][e];
        }
    }
}

// part[chunk][t][ci][co] = sum over the chunk's rows (n, s) of x[n, nbr[s, t], ci] dy[n, s, co]
// (grid (27, nchunk), 8 warps: warp w takes input-channel tile w & 1 (16 channels) and
// output-channel tile w >> 1 (8 channels); rows staged 32 at a time).
__global__ void __launch_bounds__(256)
k_conv_bwd_w_tc(int NS, int S, int Cin, int Cout, const float *__restrict__ x, const float *__restrict__ dy,
                const int32_t *__restrict__ nbr, int rows_per_chunk, float *__restrict__ part) {
    __shared__ float xs[32][kMaxCh + 1];
    __shared__ float gs[32][kMaxCh + 1];
    const int t = blockIdx.x, chunk = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const int mt = warp & 1, nt = warp >> 1;
    const bool live = 16 * mt < Cin && 8 * nt < Cout;
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int r0 = chunk * rows_per_chunk, r1 = min(NS, r0 + rows_per_chunk);
    for (int rb = r0; rb < r1; rb += 32) {
        __syncthreads();
        for (int i = threadIdx.x; i < 32 * kMaxCh; i += blockDim.x) {
            const int rr = i / kMaxCh, c = i % kMaxCh;
            const int row = rb + rr;
            float xv = 0.f, gv = 0.f;
            if (row < r1) {
                const int n = row / S, s = row % S;
                const int src = nbr[s * 27 + t];
                if (c < Cin && src >= 0) xv = x[((int64_t)n * S + src) * Cin + c];
                if (c < Cout) gv = dy[(int64_t)row * Cout + c];
            }
            xs[rr][c] = xv;
            gs[rr][c] = gv;
        }
        __syncthreads();
        if (!live) continue;
#pragma unroll
        for (int kk = 0; kk < 32; kk += 16) {
            uint32_t ah[4], al[4], bh[2], bl[2];
            const int ca = 16 * mt + g, cb = ca + 8;      // A rows (m) = input channels
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {             // A columns (k) = rows kk + 2q (+8)
                const int rr = kk + 2 * q + 8 * hh;
                split2(xs[rr][ca], xs[rr + 1][ca], ah[2 * hh], al[2 * hh]);
                split2(xs[rr][cb], xs[rr + 1][cb], ah[2 * hh + 1], al[2 * hh + 1]);
                const int co = 8 * nt + g;                // B column (n) = output channel
                split2(gs[rr][co], gs[rr + 1][co], bh[hh], bl[hh]);
            }
            mma16816(d, ah, bh[0], bh[1]);
            mma16816(d, ah, bl[0], bl[1]);
            mma16816(d, al, bh[0], bh[1]);
        }
    }
    if (!live) return;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int ci = 16 * mt + g + (e < 2 ? 0 : 8), co = 8 * nt + 2 * q + (e & 1);
        if (ci < Cin && co < Cout) part[(((int64_t)chunk * 27 + t) * Cin + ci) * Cout + co] = d[e];
    }
}

// gW = sum over chunks (fixed order); gb[co] = sum over rows of dy.
__global__ void k_conv_reduce(int nchunk, int nw, const float *__restrict__ part, float *__restrict__ gW) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    float a = 0.f;
    for (int c = 0; c < nchunk; ++c) a += part[(int64_t)c * nw + i];
    gW[i] = a;
}
__global__ void k_bias_grad(int NS, int Cout, const float *__restrict__ dy, float *__restrict__ gb) {
    __shared__ float red[256];
    const int co = blockIdx.x;
    float a = 0.f;
    for (int r = threadIdx.x; r < NS; r += blockDim.x) a += dy[(int64_t)r * Cout + co];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[co] = red[0];
}

__global__ void k_relu_mask(int64_t n, const float *__restrict__ z, float *__restrict__ g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(z[i] > 0.f)) g[i] = 0.f;
}

// Per-sample relative squared error and its gradient; loss[n] written.
__global__ void k_loss(int S, int N, const float *__restrict__ out, const float *__restrict__ tgt,
                       float *__restrict__ dout, float *__restrict__ loss) {
    __shared__ float r1[256], r2[256];
    const int n = blockIdx.x;
    float a = 0.f, d = 0.f;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const float e = out[(int64_t)n * S + s] - tgt[(int64_t)n * S + s];
        const float y = tgt[(int64_t)n * S + s];
        a += e * e;
        d += y * y;
    }
    r1[threadIdx.x] = a;
    r2[threadIdx.x] = d;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] += r2[threadIdx.x + o];
        }
        __syncthreads();
    }
    const float den = r2[0] > 0.f ? r2[0] : 1.f;
    for (int s = threadIdx.x; s < S; s += blockDim.x)
        dout[(int64_t)n * S + s] = 2.f * (out[(int64_t)n * S + s] - tgt[(int64_t)n * S + s]) / (den * N);
    if (threadIdx.x == 0) loss[n] = r1[0] / den;
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, float lr, float b1, float b2, float c1,
                       float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
}

// ---- training data --------------------------------------------------------------------------
// u in [-1, 1) from splitmix64(seed), element i = output i+1 of the stream.
__global__ void k_uniform(uint64_t seed, int64_t count, double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
}

// C = A B with A (M x K) and B (K x N), both column-major, FP64; 64 x 64 tiles.
__global__ void __launch_bounds__(256)
k_dgemm(int M, int N, int K, const double *__restrict__ A, const double *__restrict__ B, double *__restrict__ C) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = i / 64, mm = i % 64;
            As[kk][mm] = (m0 + mm < M && k0 + kk < K) ? A[(int64_t)(k0 + kk) * M + m0 + mm] : 0.0;
            const int nn = i / 16, k2 = i % 16;
            Bs[k2][nn] = (n0 + nn < N && k0 + k2 < K) ? B[(int64_t)(n0 + nn) * K + k0 + k2] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            if (m < M && n < N) C[(int64_t)n * M + m] = acc[i][j];
        }
}

// Scaled FP32 training pairs: X = rho / ||rho||, Y = t * d / ||rho|| (sample per CTA).
__global__ void k_scale_pairs(int S, const double *__restrict__ R, const double *__restrict__ T, double d,
                              float *__restrict__ X, float *__restrict__ Y) {
    __shared__ double red[256];
    const int n = blockIdx.x;
    double a = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) a += R[(int64_t)n * S + s] * R[(int64_t)n * S + s];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double nr = sqrt(red[0]);
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        X[(int64_t)n * S + s] = (float)(R[(int64_t)n * S + s] * inv);
        Y[(int64_t)n * S + s] = (float)(T[(int64_t)n * S + s] * d * inv);
    }
}

// ---- in-apply stage ------------------------------------------------------------------------
// rho = zsave - C y2 + work2[tail] (work2[tail] holds E (LU)^{-1} F y2); x0 = rho / ||rho||.
template <typename VT>
__global__ void __launch_bounds__(1024)
k_learned_rho(int S, int64_t e, const VT *__restrict__ work, const VT *__restrict__ work2,
              const VT *__restrict__ zsave, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
              const VT *__restrict__ v, float *__restrict__ x0, float *__restrict__ rnorm) {
    __shared__ float red[1024];
    float a = 0.f;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        VT cy = 0;
        for (int64_t p = rp[s]; p < rp[s + 1]; ++p) cy += v[p] * work[e + ci[p]];
        const float r = (float)(zsave[s] - cy + work2[e + s]);
        x0[s] = r;
        a += r * r;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float nr = sqrtf(red[0]);
    const float inv = nr > 0.f ? 1.f / nr : 0.f;
    for (int s = threadIdx.x; s < S; s += blockDim.x) x0[s] *= inv;
    if (threadIdx.x == 0) *rnorm = nr;
}

// y2 += (||rho|| / d) * out
template <typename VT>
__global__ void k_learned_update(int S, int64_t e, const float *__restrict__ out, const float *__restrict__ rnorm,
                                 double d, VT *__restrict__ work) {
    const float sc = (float)(*rnorm / d);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) work[e + s] += (VT)(sc * out[s]);
}

template <typename VT>
__global__ void k_cast_out(int64_t n, const VT *__restrict__ src, double *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

template <typename VT>
__global__ void k_copy_vec(int64_t n, const VT *__restrict__ src, VT *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

// ---- host: network passes ----------------------------------------------------------------------
// Tensor cores for the C -> C layers (both channel counts >= 8).
static bool conv_tc(const NetDev &net, int l) { return net.cin[l] >= 8 && net.cout[l] >= 8; }
static size_t conv_tc_smem(const NetDev &net, int l) { return (size_t)27 * net.cin[l] * net.cout[l] * 2; }

static void launch_conv_fwd(const NetDev &net, int l, int N, const float *in, float *z, float *h, int relu,
                            cudaStream_t st) {
    if (conv_tc(net, l)) {
        const int sites = 16 * kConvTcWarps;
        k_conv_fwd_tc<<<dim3((net.S + sites - 1) / sites, N), 32 * kConvTcWarps, conv_tc_smem(net, l), st>>>(
            net.S, net.cin[l], net.cout[l], in, net.Wb[l], net.b[l], net.nbr, z, h, relu);
    } else {
        dim3 grid((net.S + kConvSitesPerCta - 1) / kConvSitesPerCta, N), block(32, 8);
        k_conv_fwd<<<grid, block, 0, st>>>(net.S, net.cin[l], net.cout[l], in, net.Wb[l], net.b[l], net.nbr, z, h, relu);
    }
    count_launch();
}

void net_forward(NetDev &net, int N, const float *x0, float *const zs[4], float *const hs[3], cudaStream_t st) {
    const float *in = x0;
    for (int l = 0; l < kNetLayers; ++l) {
        launch_conv_fwd(net, l, N, in, zs[l], l < 3 ? hs[l] : nullptr, l < 3 ? 1 : 0, st);
        if (l < 3) in = hs[l];
    }
}

// Backward from dout (N x S) through the stored activations; gradients into net.gW/gb.
void net_backward(NetDev &net, int N, const float *x0, float *const zs[4], float *const hs[3], float *dout,
                  float *gbuf0, float *gbuf1, float *part, int nchunk, cudaStream_t st) {
    const int NS = N * net.S;
    const int rows = (NS + nchunk - 1) / nchunk;
    float *g = dout;
    for (int l = kNetLayers - 1; l >= 0; --l) {
        if (l < 3) {
            k_relu_mask<<<1216, 256, 0, st>>>((int64_t)NS * net.cout[l], zs[l], g);
            count_launch();
        }
        const float *inp = l == 0 ? x0 : hs[l - 1];
        const int nw = 27 * net.cin[l] * net.cout[l];
        if (conv_tc(net, l))
            k_conv_bwd_w_tc<<<dim3(27, nchunk), 256, 0, st>>>(NS, net.S, net.cin[l], net.cout[l], inp, g, net.nbr,
                                                              rows, part);
        else
            k_conv_bwd_w<<<dim3(27, nchunk), dim3(32, 8), 0, st>>>(NS, net.S, net.cin[l], net.cout[l], inp, g, net.nbr,
                                                                 rows, part);
        k_conv_reduce<<<(nw + 255) / 256, 256, 0, st>>>(nchunk, nw, part, net.gW[l]);
        k_bias_grad<<<net.cout[l], 256, 0, st>>>(NS, net.cout[l], g, net.gb[l]);
        count_launch(3);
        if (l > 0) {
            float *dx = (g == gbuf0) ? gbuf1 : gbuf0;
            if (conv_tc(net, l)) {
                const int sites = 16 * kConvTcWarps;
                k_conv_bwd_data_tc<<<dim3((net.S + sites - 1) / sites, N), 32 * kConvTcWarps,
                                     conv_tc_smem(net, l), st>>>(net.S, net.cin[l], net.cout[l], g, net.Wb[l], net.nbr,
                                                                 dx);
            } else {
                dim3 grid((net.S + kConvSitesPerCta - 1) / kConvSitesPerCta, N), block(32, 8);
                k_conv_bwd_data<<<grid, block, 0, st>>>(net.S, net.cin[l], net.cout[l], g, net.Wb[l], net.nbr, dx);
            }
            count_launch();
            g = dx;
        }
    }
}

void net_adam(NetDev &net, float lr, cudaStream_t st) {
    net.adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net.adam_t), c2 = 1.f - powf(b2, (float)net.adam_t);
    for (int l = 0; l < kNetLayers; ++l) {
        const int64_t nw = 27LL * net.cin[l] * net.cout[l];
        k_adam<<<256, 256, 0, st>>>(nw, net.W[l], net.gW[l], net.mW[l], net.vW[l], net.Wb[l], lr, b1, b2, c1, c2);
        k_adam<<<1, 256, 0, st>>>(net.cout[l], net.b[l], net.gb[l], net.mb[l], net.vb[l], nullptr, lr, b1, b2, c1, c2);
        count_launch(2);
    }
}

void net_kernels_init() {
    const int bytes = 27 * kMaxCh * kMaxCh * 2;          // all taps of a 32 -> 32 layer in BF16
    GEMSLR_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GEMSLR_CUDA(cudaFuncSetAttribute(k_conv_bwd_data_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

void net_sync_bf16(NetDev &net, cudaStream_t st) {
    for (int l = 0; l < kNetLayers; ++l) {
        k_to_bf16<<<256, 256, 0, st>>>(27LL * net.cin[l] * net.cout[l], net.W[l], net.Wb[l]);
        count_launch();
    }
}

void launch_uniform(uint64_t seed, int64_t count, double *out, cudaStream_t st) {
    k_uniform<<<1216, 256, 0, st>>>(seed, count, out);
    count_launch();
}

void launch_dgemm(int M, int N, int K, const double *A, const double *B, double *C, cudaStream_t st) {
    dim3 grid((M + 63) / 64, (N + 63) / 64);
    k_dgemm<<<grid, 256, 0, st>>>(M, N, K, A, B, C);
    count_launch();
}

void launch_scale_pairs(int S, int count, const double *R, const double *T, double d, float *X, float *Y,
                        cudaStream_t st) {
    k_scale_pairs<<<count, 256, 0, st>>>(S, R, T, d, X, Y);
    count_launch();
}

void launch_loss(int S, int N, const float *out, const float *tgt, float *dout, float *loss, cudaStream_t st) {
    k_loss<<<N, 256, 0, st>>>(S, N, out, tgt, dout, loss);
    count_launch();
}

template <typename VT>
void learned_save(const LearnedStage<VT> &L, int64_t e, const VT *work, cudaStream_t st) {
    k_copy_vec<VT><<<(L.net->S + 255) / 256, 256, 0, st>>>(L.net->S, work + e, L.zsave);
    count_launch();
}

template <typename VT>
void learned_rho_and_update(const LearnedStage<VT> &L, int64_t e, VT *work, cudaStream_t st) {
    NetDev &net = *L.net;
    k_learned_rho<VT><<<1, 1024, 0, st>>>(net.S, e, work, L.work2, L.zsave, L.C_rp, L.C_ci, L.C_v, L.act0, L.rnorm);
    count_launch();
    float *zs[4] = {L.act1, L.act2, L.act1, L.act2};
    float *hs[3] = {L.act1, L.act2, L.act1};
    // forward with ping-pong buffers (no backward here): layer l reads hs[l-1], writes zs/hs in place
    const float *in = L.act0;
    float *bufs[2] = {L.act1, L.act2};
    for (int l = 0; l < kNetLayers; ++l) {
        float *o = bufs[l & 1];
        launch_conv_fwd(net, l, 1, in, o, nullptr, 0, st);
        if (l < 3) {
            k_relu_mask<<<(net.S * net.cout[l] + 255) / 256, 256, 0, st>>>((int64_t)net.S * net.cout[l], o, o);
            count_launch();
        }
        in = o;
    }
    (void)zs;
    (void)hs;
    k_learned_update<VT><<<(net.S + 255) / 256, 256, 0, st>>>(net.S, e, in, L.rnorm, net.dscale, work);
    count_launch();
}

template <typename VT>
void launch_cast_out(int64_t n, const VT *src, double *dst, cudaStream_t st) {
    if (n <= 0) return;
    k_cast_out<VT><<<(unsigned)std::min<int64_t>((n + 255) / 256, 4864), 256, 0, st>>>(n, src, dst);
    count_launch();
}
template void launch_cast_out<double>(int64_t, const double *, double *, cudaStream_t);
template void launch_cast_out<float>(int64_t, const float *, double *, cudaStream_t);

template void learned_save<double>(const LearnedStage<double> &, int64_t, const double *, cudaStream_t);
template void learned_save<float>(const LearnedStage<float> &, int64_t, const float *, cudaStream_t);
template void learned_rho_and_update<double>(const LearnedStage<double> &, int64_t, double *, cudaStream_t);
template void learned_rho_and_update<float>(const LearnedStage<float> &, int64_t, float *, cudaStream_t);

}  // namespace gemslr
