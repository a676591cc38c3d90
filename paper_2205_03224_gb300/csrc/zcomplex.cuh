// Complex FP64 scalar of the complex-shifted hierarchy (Sec. 5.2.3): the
// diagonal blocks are factored as B + i alpha I, so their factors, the
// low-rank terms and every vector of the application are complex.  A plain
// 16-byte {re, im} pair with the arithmetic the substitution, coupling and
// Krylov kernels need; the default constructor is trivial so that the type
// can live in shared memory.
#pragma once

#include <cuda_runtime.h>

namespace gemslr {

struct __align__(16) zc {
    double re, im;
    zc() = default;
    __host__ __device__ constexpr zc(double r) : re(r), im(0.0) {}
    __host__ __device__ constexpr zc(double r, double i) : re(r), im(i) {}
};

__host__ __device__ __forceinline__ zc operator+(zc a, zc b) { return zc(a.re + b.re, a.im + b.im); }
__host__ __device__ __forceinline__ zc operator-(zc a, zc b) { return zc(a.re - b.re, a.im - b.im); }
__host__ __device__ __forceinline__ zc operator-(zc a) { return zc(-a.re, -a.im); }
__host__ __device__ __forceinline__ zc operator*(zc a, zc b) {
    return zc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__host__ __device__ __forceinline__ zc operator*(double a, zc b) { return zc(a * b.re, a * b.im); }
__host__ __device__ __forceinline__ zc &operator+=(zc &a, zc b) { a = a + b; return a; }
__host__ __device__ __forceinline__ zc &operator-=(zc &a, zc b) { a = a - b; return a; }
__host__ __device__ __forceinline__ zc &operator*=(zc &a, zc b) { a = a * b; return a; }
__host__ __device__ __forceinline__ bool operator==(zc a, zc b) { return a.re == b.re && a.im == b.im; }
__host__ __device__ __forceinline__ zc conj(zc a) { return zc(a.re, -a.im); }
__host__ __device__ __forceinline__ double abs2(zc a) { return a.re * a.re + a.im * a.im; }

template <typename T> struct IsComplex { static constexpr bool value = false; };
template <> struct IsComplex<zc> { static constexpr bool value = true; };

// Element type of the user-side vectors a substitution reads (`in`) and
// writes (`out_final`): FP64 for the real hierarchies, complex for zc.
template <typename VT> struct IoOf { using type = double; };
template <> struct IoOf<zc> { using type = zc; };
template <typename VT> using IoT = typename IoOf<VT>::type;

#ifdef __CUDACC__
// Warp shuffles and L2-only loads, generic and for zc (two 8-byte halves).
template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int o, int width = 32) { return __shfl_xor_sync(0xffffffffu, v, o, width); }
template <>
__device__ __forceinline__ zc shfl_xor<zc>(zc v, int o, int width) {
    return zc(__shfl_xor_sync(0xffffffffu, v.re, o, width), __shfl_xor_sync(0xffffffffu, v.im, o, width));
}
template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <> __device__ __forceinline__ zc ldcg<zc>(const zc *p) {
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return zc(v.x, v.y);
}
#endif

}  // namespace gemslr
