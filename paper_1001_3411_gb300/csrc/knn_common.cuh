// Device helpers shared by the two kNN kernels (knn.cu: P lanes per query;
// knn32.cu: one query per lane): histogram bins of squared distances, the M4
// kernel, cell ranges of the Morton-sorted particles and the periodic
// minimum-image difference.
#pragma once

#include "hop_internal.cuh"

namespace {

// 1/8-octave bin of v relative to tau's own bin: bins 0..31, bin 31 holds
// tau's octave-eighth, lower bins smaller values; bin 0 also holds everything
// below.  Monotone in v for v >= 0.
__device__ __forceinline__ int bin_base(float tau) { return (int)(__float_as_uint(tau) >> 20); }
__device__ __forceinline__ int bin_base(double tau)
{
    return (int)((unsigned long long)__double_as_longlong(tau) >> 49);
}
__device__ __forceinline__ int bin_of(float v, int tb)
{
    int b = (int)(__float_as_uint(v) >> 20) - tb + (kHistBins - 1);
    return min(max(b, 0), kHistBins - 1);
}
__device__ __forceinline__ int bin_of(double v, int tb)
{
    int b = (int)((unsigned long long)__double_as_longlong(v) >> 49) - tb + (kHistBins - 1);
    return min(max(b, 0), kHistBins - 1);
}
// Largest value whose bin is <= b (b < 31), or -1 if that is below zero.
__device__ __forceinline__ float bin_upper(float, int tb, int b)
{
    int e = tb - (kHistBins - 1) + b + 1;
    if (e <= 0) return -1.f;
    return __uint_as_float(((uint32_t)e << 20) - 1u);
}
__device__ __forceinline__ double bin_upper(double, int tb, int b)
{
    long long e = (long long)tb - (kHistBins - 1) + b + 1;
    if (e <= 0) return -1.0;
    return __longlong_as_double((long long)(((unsigned long long)e << 49) - 1ull));
}

// M4 cubic spline w(q) (Monaghan & Lattanzio 1985): W = w(r/h) / (pi h^3).
template <typename T> __device__ __forceinline__ T m4(T q)
{
    if (q < T(1)) return T(1) - T(1.5) * q * q + T(0.75) * q * q * q;
    if (q < T(2)) {
        T t = T(2) - q;
        return T(0.25) * t * t * t;
    }
    return T(0);
}

// Contiguous range of sorted particles in level-l cell `code`.
__device__ __forceinline__ void cell_range(const uint32_t *__restrict__ cellT,
                                           const uint64_t *__restrict__ keys, int Ld, int l,
                                           uint64_t code, uint32_t &a, uint32_t &b)
{
    if (l <= Ld) {
        const int sh = 3 * (Ld - l);
        a = cellT[code << sh];
        b = cellT[(code + 1) << sh];
        return;
    }
    const int up = 3 * (l - Ld);
    const uint64_t pc = code >> up;
    uint32_t lo = cellT[pc], hi = cellT[pc + 1];
    const int ksh = 3 * (kMaxLevel - l);
    const uint64_t k0 = code << ksh, k1 = (code + 1) << ksh;
    // lower_bound(k0)
    uint32_t L = lo, H = hi;
    while (L < H) {
        uint32_t m = (L + H) >> 1;
        if (keys[m] < k0) L = m + 1; else H = m;
    }
    a = L;
    H = hi;
    while (L < H) {
        uint32_t m = (L + H) >> 1;
        if (keys[m] < k1) L = m + 1; else H = m;
    }
    b = L;
}

template <typename T> __device__ __forceinline__ T wrapdiff(T xj, T xi, T box, T half)
{
    // Minimum-image difference with one rounding: the coordinate >= L/2 of
    // the pair is moved by -L (exact) when the plain difference exceeds L/2.
    T d = xj - xi;
    if (d > half) return (xj - box) - xi;
    if (d < -half) return xj - (xi - box);
    return d;
}

}  // namespace
