// Rayleigh quotient of the randomized set-up of the low-rank corrections:
// B = V^T Z for two s x b column-major FP64 blocks (b <= kMaxCols).  One CTA
// per (column c of Z, group of 8 columns of V): eight dot products over s,
// each thread summing a strided share and the CTA reducing in a fixed order,
// so B is the same from run to run.
#include "device.h"
#include "ptx.cuh"

namespace gemslr {

namespace {

constexpr int kGramThreads = 256;

__global__ void __launch_bounds__(kGramThreads)
k_gram(int64_t s, int b, const double *__restrict__ V, const double *__restrict__ Z, double *__restrict__ B) {
    __shared__ double red[8][kGramThreads / 32];
    const int c = blockIdx.x, j0 = 8 * blockIdx.y;
    const double *z = Z + (int64_t)c * s;
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < s; i += blockDim.x) {
        const double zi = z[i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (j0 + q < b) acc[q] += V[(int64_t)(j0 + q) * s + i] * zi;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double t = warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < 8 && j0 + (int)threadIdx.x < b) {
        double t = 0.0;
        for (int w = 0; w < kGramThreads / 32; ++w) t += red[threadIdx.x][w];
        B[(int64_t)c * b + j0 + threadIdx.x] = t;     // B[j, c], column-major b x b
    }
}

}  // namespace

void launch_gram(int64_t s, int b, const double *V, const double *Z, double *B, cudaStream_t st) {
    if (b <= 0) return;
    k_gram<<<dim3(b, (b + 7) / 8), kGramThreads, 0, st>>>(s, b, V, Z, B);
    count_launch();
}

}  // namespace gemslr
