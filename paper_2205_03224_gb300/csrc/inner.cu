// Inner GMRES at the root level (Alg. 2 step 9).
//
// Instead of the single application y2 = M_S^-1 z2 (eq. gemslr6 and the levels
// below), the root level solves S_hat_0 y2 = z2 by k steps of GMRES from
// y2 = 0, right preconditioned by M_S^-1, with the inexact Schur complement
// S_hat_0 = C_0 - E_0 U^-1 L^-1 F_0 of Sec. 2.4.  One product S_hat_0 z is one
// level-0 substitution and one pass over the tail rows of A_hat:
//   t = [ -U^-1 L^-1 F_0 z ; z ]   (the level-0 up sweep on a zero level part)
//   S_hat_0 z = (A_hat t)[e0:n]    (the rows of E_0 meet -U^-1 L^-1 F_0 z, the rows of C_0 meet z)
// The Arnoldi vectors have the tail length; they are orthogonalised by
// classical Gram-Schmidt with a second pass (two reductions per step), with
// FP64 sums whatever the vector type.  Each reduction is per-CTA partials
// finished by the last CTA in a fixed order (deterministic).  Kernels of a
// step that follows a happy breakdown return at once.
#include <cmath>

#include "device.h"
#include "ptx.cuh"

namespace gemslr {

namespace {

constexpr int kIT = kReduceThreads;            // threads of every inner kernel
constexpr int kSlots = kMaxInner + 2;          // partial slots: j + 1 dots and a squared norm
constexpr int kLdh = kMaxInner + 1;            // leading dimension of H

// acc[s] summed over the CTA, written to partial[s * gridDim.x + blockIdx.x] for s < ns.
__device__ __forceinline__ void cta_partials(const double (&acc)[kSlots], int ns, double *partial) {
    __shared__ double red[kSlots][kIT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        if (s < ns) {
            const double v = warp_sum(acc[s]);
            if (lane == 0) red[s][warp] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kIT / 32; ++q) t += red[threadIdx.x][q];
        partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// True in the CTA that finishes last (its partials see everyone's).
__device__ bool last_cta(unsigned *counter) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// beta = ||z2||; resets the step state.
template <typename VT>
__global__ void __launch_bounds__(kIT) k_inner_norm(const InnerView<VT> iv, const VT *__restrict__ z2) {
    __shared__ double tot[kSlots];
    double acc[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) acc[s] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.m; i += (int64_t)gridDim.x * kIT) {
        const double z = (double)z2[i];
        acc[0] = fma(z, z, acc[0]);
    }
    cta_partials(acc, 1, iv.partial);
    if (!last_cta(iv.counter)) return;
    reduce_columns<double>(iv.partial, (int)gridDim.x, 1, tot);
    if (threadIdx.x == 0) {
        const double beta = sqrt(tot[0]);
        iv.ctl->beta = beta;
        iv.ctl->done = beta == 0.0 ? 1 : 0;
        iv.ctl->steps = 0;
        iv.ctl->wn0 = 0.0;
        *iv.counter = 0u;
    }
}

// v_0 = z2 / beta into V[:, 0] and the tail of work2; the level part of work2
// is cleared for the first S_hat product.
template <typename VT>
__global__ void __launch_bounds__(kIT) k_inner_start(const InnerView<VT> iv, const VT *__restrict__ z2,
                                                     VT *__restrict__ work2) {
    const double beta = iv.ctl->beta;
    const double s = beta > 0.0 ? 1.0 / beta : 0.0;
    const int64_t stride = (int64_t)gridDim.x * kIT;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.m; i += stride) {
        const VT v = (VT)((double)z2[i] * s);
        iv.V[i] = v;
        work2[iv.e0 + i] = v;
    }
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.e0; i += stride) work2[i] = (VT)0;
}

// Step j: z_j = tail of work2 (saved into Z[:, j]); w = (A_hat work2)[e0:n] =
// S_hat_0 z_j; first-pass coefficients h_c = v_c . w (c <= j) into H[:, j] and
// ||w|| into wn0.
template <typename VT>
__global__ void __launch_bounds__(kIT) k_inner_spmv_dots(const InnerView<VT> iv, int j,
                                                         const VT *__restrict__ work2) {
    __shared__ double tot[kSlots];
    if (iv.ctl->done) return;
    double acc[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) acc[s] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.m; i += (int64_t)gridDim.x * kIT) {
        const int64_t pa = iv.rp[i], pb = iv.rp[i + 1];
        VT y = 0;
        for (int64_t p = pa; p < pb; ++p) y += iv.v[p] * work2[iv.ci[p]];
        iv.w[i] = y;
        iv.Z[(int64_t)j * iv.m + i] = work2[iv.e0 + i];
        const double yd = (double)y;
#pragma unroll
        for (int c = 0; c <= kMaxInner; ++c)
            if (c <= j) acc[c] = fma((double)iv.V[(int64_t)c * iv.m + i], yd, acc[c]);
        acc[kSlots - 1] = fma(yd, yd, acc[kSlots - 1]);
    }
    // slot j + 1 carries w . w (moved from the last slot; j + 1 <= kMaxInner)
#pragma unroll
    for (int s = 1; s < kSlots - 1; ++s)
        if (s == j + 1) acc[s] = acc[kSlots - 1];
    cta_partials(acc, j + 2, iv.partial);
    if (!last_cta(iv.counter)) return;
    reduce_columns<double>(iv.partial, (int)gridDim.x, j + 2, tot);
    if (threadIdx.x <= j) iv.H[threadIdx.x + (int64_t)j * kLdh] = tot[threadIdx.x];
    if (threadIdx.x == 0) {
        iv.ctl->wn0 = sqrt(tot[j + 1]);
        *iv.counter = 0u;
    }
}

// Step j, second pass: w -= V h (first-pass coefficients), then h2_c = v_c . w
// and ||w||^2; H[:, j] += h2, h_{j+1,j} = sqrt(||w||^2 - ||h2||^2) (the norm
// after the second projection), and the happy-breakdown test
// h_{j+1,j} <= 1e-14 ||S_hat z_j||.
template <typename VT>
__global__ void __launch_bounds__(kIT) k_inner_sub_dots(const InnerView<VT> iv, int j) {
    __shared__ double tot[kSlots];
    if (iv.ctl->done) return;
    double h[kMaxInner + 1];
#pragma unroll
    for (int c = 0; c <= kMaxInner; ++c) h[c] = c <= j ? iv.H[c + (int64_t)j * kLdh] : 0.0;
    double acc[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) acc[s] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.m; i += (int64_t)gridDim.x * kIT) {
        double vc[kMaxInner + 1];
#pragma unroll
        for (int c = 0; c <= kMaxInner; ++c) vc[c] = c <= j ? (double)iv.V[(int64_t)c * iv.m + i] : 0.0;
        double x = (double)iv.w[i];
#pragma unroll
        for (int c = 0; c <= kMaxInner; ++c) x = fma(-vc[c], h[c], x);
        const VT xv = (VT)x;
        iv.w[i] = xv;
        const double xd = (double)xv;
#pragma unroll
        for (int c = 0; c <= kMaxInner; ++c)
            if (c <= j) acc[c] = fma(vc[c], xd, acc[c]);
        acc[kSlots - 1] = fma(xd, xd, acc[kSlots - 1]);
    }
#pragma unroll
    for (int s = 1; s < kSlots - 1; ++s)
        if (s == j + 1) acc[s] = acc[kSlots - 1];
    cta_partials(acc, j + 2, iv.partial);
    if (!last_cta(iv.counter)) return;
    reduce_columns<double>(iv.partial, (int)gridDim.x, j + 2, tot);
    if (threadIdx.x <= j) {
        const double h2 = tot[threadIdx.x];
        iv.ctl->h2[threadIdx.x] = h2;
        iv.H[threadIdx.x + (int64_t)j * kLdh] += h2;
    }
    if (threadIdx.x == 0) {
        double hh = 0.0;
        for (int c = 0; c <= j; ++c) hh = fma(tot[c], tot[c], hh);
        const double hn = sqrt(fmax(tot[j + 1] - hh, 0.0));
        iv.H[j + 1 + (int64_t)j * kLdh] = hn;
        iv.ctl->steps = j + 1;
        if (!(hn > 1e-14 * iv.ctl->wn0)) iv.ctl->done = 1;
        *iv.counter = 0u;
    }
}

// Step j, closing: v_{j+1} = (w - V h2) / h_{j+1,j} into V[:, j+1] and the tail
// of work2, and the level part of work2 cleared for the next S_hat product.
template <typename VT>
__global__ void __launch_bounds__(kIT) k_inner_scale(const InnerView<VT> iv, int j, VT *__restrict__ work2) {
    if (iv.ctl->done) return;
    double h2[kMaxInner + 1];
#pragma unroll
    for (int c = 0; c <= kMaxInner; ++c) h2[c] = c <= j ? iv.ctl->h2[c] : 0.0;
    const double inv = 1.0 / iv.H[j + 1 + (int64_t)j * kLdh];
    const int64_t stride = (int64_t)gridDim.x * kIT;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.m; i += stride) {
        double x = (double)iv.w[i];
#pragma unroll
        for (int c = 0; c <= kMaxInner; ++c)
            if (c <= j) x = fma(-(double)iv.V[(int64_t)c * iv.m + i], h2[c], x);
        const VT v = (VT)(x * inv);
        iv.V[(int64_t)(j + 1) * iv.m + i] = v;
        work2[iv.e0 + i] = v;
    }
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.e0; i += stride) work2[i] = (VT)0;
}

// min || beta e_1 - H c || over the first `steps` columns: Givens rotations
// reduce H to upper-triangular form, then back substitution (one thread).
__global__ void k_inner_lsq(InnerCtl *ctl, const double *Hg) {
    if (threadIdx.x != 0) return;
    const int n = ctl->steps;
    double H[kLdh * kMaxInner], g[kLdh], cs[kMaxInner], sn[kMaxInner], c[kMaxInner];
    for (int q = 0; q < kLdh * kMaxInner; ++q) H[q] = Hg[q];
    for (int q = 0; q < kLdh; ++q) g[q] = 0.0;
    g[0] = ctl->beta;
    for (int jj = 0; jj < n; ++jj) {
        double *col = H + jj * kLdh;
        for (int i = 0; i < jj; ++i) {
            const double t = cs[i] * col[i] + sn[i] * col[i + 1];
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
            col[i] = t;
        }
        const double den = hypot(col[jj], col[jj + 1]);
        cs[jj] = den > 0.0 ? col[jj] / den : 1.0;
        sn[jj] = den > 0.0 ? col[jj + 1] / den : 0.0;
        col[jj] = den;
        col[jj + 1] = 0.0;
        g[jj + 1] = -sn[jj] * g[jj];
        g[jj] = cs[jj] * g[jj];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = g[i];
        for (int q = i + 1; q < n; ++q) t -= H[i + q * kLdh] * c[q];
        c[i] = t / H[i + i * kLdh];
    }
    for (int i = 0; i < kMaxInner; ++i) ctl->c[i] = i < n ? c[i] : 0.0;
}

// y2 = sum_j c_j z_j into the tail of work (and of out_final, as FP64).
template <typename VT>
__global__ void __launch_bounds__(kIT) k_inner_combine(const InnerView<VT> iv, VT *__restrict__ work,
                                                       double *__restrict__ out_final) {
    double c[kMaxInner];
    const int n = iv.ctl->steps;
#pragma unroll
    for (int q = 0; q < kMaxInner; ++q) c[q] = q < n ? iv.ctl->c[q] : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kIT + threadIdx.x; i < iv.m; i += (int64_t)gridDim.x * kIT) {
        double y = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxInner; ++q)
            if (q < n) y = fma(c[q], (double)iv.Z[(int64_t)q * iv.m + i], y);
        const VT yv = (VT)y;
        work[iv.e0 + i] = yv;
        if (out_final) out_final[iv.e0 + i] = (double)yv;
    }
}

}  // namespace

template <typename VT>
void launch_inner_norm(const InnerView<VT> &iv, const VT *z2, cudaStream_t st) {
    k_inner_norm<VT><<<iv.grid, kIT, 0, st>>>(iv, z2); count_launch();
}
template <typename VT>
void launch_inner_start(const InnerView<VT> &iv, const VT *z2, VT *work2, cudaStream_t st) {
    k_inner_start<VT><<<iv.grid, kIT, 0, st>>>(iv, z2, work2); count_launch();
}
template <typename VT>
void launch_inner_spmv_dots(const InnerView<VT> &iv, int j, const VT *work2, cudaStream_t st) {
    k_inner_spmv_dots<VT><<<iv.grid, kIT, 0, st>>>(iv, j, work2); count_launch();
}
template <typename VT>
void launch_inner_sub_dots(const InnerView<VT> &iv, int j, cudaStream_t st) {
    k_inner_sub_dots<VT><<<iv.grid, kIT, 0, st>>>(iv, j); count_launch();
}
template <typename VT>
void launch_inner_scale(const InnerView<VT> &iv, int j, VT *work2, cudaStream_t st) {
    k_inner_scale<VT><<<iv.grid, kIT, 0, st>>>(iv, j, work2); count_launch();
}
template <typename VT>
void launch_inner_lsq(const InnerView<VT> &iv, cudaStream_t st) {
    k_inner_lsq<<<1, 32, 0, st>>>(iv.ctl, iv.H); count_launch();
}
template <typename VT>
void launch_inner_combine(const InnerView<VT> &iv, VT *work, double *out_final, cudaStream_t st) {
    k_inner_combine<VT><<<iv.grid, kIT, 0, st>>>(iv, work, out_final); count_launch();
}

#define GEMSLR_INNER_INST(VT)                                                                               \
    template void launch_inner_norm<VT>(const InnerView<VT> &, const VT *, cudaStream_t);                  \
    template void launch_inner_start<VT>(const InnerView<VT> &, const VT *, VT *, cudaStream_t);           \
    template void launch_inner_spmv_dots<VT>(const InnerView<VT> &, int, const VT *, cudaStream_t);        \
    template void launch_inner_sub_dots<VT>(const InnerView<VT> &, int, cudaStream_t);                     \
    template void launch_inner_scale<VT>(const InnerView<VT> &, int, VT *, cudaStream_t);                  \
    template void launch_inner_lsq<VT>(const InnerView<VT> &, cudaStream_t);                               \
    template void launch_inner_combine<VT>(const InnerView<VT> &, VT *, double *, cudaStream_t);
GEMSLR_INNER_INST(double)
GEMSLR_INNER_INST(float)
#undef GEMSLR_INNER_INST

}  // namespace gemslr
