// Register-resident DFTs of compile-time length (FP32 demag path).
//
// dif<N, DIR, HALF>(v) transforms the N complex values a thread holds in
// registers by decimation in frequency (radix-2 split down to 8-, 4- or
// 2-point kernels), leaving X[k] at register position dif_pos<N>(k) (a
// compile-time permutation, so reordering costs nothing).  HALF = true
// declares the upper half of the input zero (the zero-padded half of a
// line), which turns the first butterfly level into a copy and a twiddle.
// Twiddle constants exp(DIR 2 pi i k / N) are evaluated at compile time by
// cos2pi / sin2pi: exact octant reduction of the rational angle k / N, then
// the Taylor series on [0, pi/4] in double, rounded to the element type.
#pragma once

#include "mm_internal.cuh"

namespace mm {

constexpr double kPiTaylor = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
    double t = x, s = x;
    for (int i = 1; i < 16; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}
constexpr double taylor_cos(double x) {
    double t = 1.0, s = 1.0;
    for (int i = 1; i < 16; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}
// cos and sin of 2 pi k / n, n a power of two
constexpr double cos2pi(int k, int n);
constexpr double sin2pi(int k, int n) {
    k = ((k % n) + n) % n;
    if (2 * k > n) return -sin2pi(n - k, n);
    if (4 * k > n) return sin2pi(n / 2 - k, n);            // sin(pi - a) = sin a
    if (8 * k > n) return cos2pi(n / 4 - k, n);            // sin a = cos(pi/2 - a)
    return taylor_sin(2.0 * kPiTaylor * k / n);
}
constexpr double cos2pi(int k, int n) {
    k = ((k % n) + n) % n;
    if (2 * k > n) return cos2pi(n - k, n);
    if (4 * k > n) return -cos2pi(n / 2 - k, n);           // cos(pi - a) = -cos a
    if (8 * k > n) return sin2pi(n / 4 - k, n);            // cos a = sin(pi/2 - a)
    return taylor_cos(2.0 * kPiTaylor * k / n);
}

// position of X[k] after dif<N>
template <int N> __host__ __device__ constexpr int dif_pos(int k) {
    if constexpr (N <= 8) {
        return k;
    } else {
        return (k & 1) ? N / 2 + dif_pos<N / 2>(k >> 1) : dif_pos<N / 2>(k >> 1);
    }
}

template <typename C> __host__ __device__ __forceinline__ C mul_dir_i(C a, int dir) {
    return dir > 0 ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// natural-order small DFTs
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft4(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = mul_dir_i(csub(v[1], v[3]), DIR);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft8(C* v) {
    using T = decltype(C{}.x);
    const T h = (T)0.70710678118654752440084436210484904;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    rdft4<DIR>(e);
    rdft4<DIR>(o);
    C w1o = cmk<C>(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
    C w2o = mul_dir_i(o[2], DIR);
    C w3o = cmk<C>(-h * (o[3].x + DIR * o[3].y), h * (DIR * o[3].x - o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1o);
    v[5] = csub(e[1], w1o);
    v[2] = cadd(e[2], w2o);
    v[6] = csub(e[2], w2o);
    v[3] = cadd(e[3], w3o);
    v[7] = csub(e[3], w3o);
}

// first DIF level: v[i] <- a + b, v[i + N/2] <- (a - b) w^i, for i = K..N/2-1
template <int N, int K, int DIR, bool HALF, typename C> __host__ __device__ __forceinline__ void dif_level(C* v) {
    if constexpr (K < N / 2) {
        using T = decltype(C{}.x);
        C a = v[K];
        C d;
        if constexpr (HALF) {
            d = a;
        } else {
            C b = v[K + N / 2];
            v[K] = cadd(a, b);
            d = csub(a, b);
        }
        if constexpr (K == 0) {
            v[K + N / 2] = d;
        } else if constexpr (4 * K == N) {
            v[K + N / 2] = mul_dir_i(d, DIR);
        } else {
            constexpr double c = cos2pi(K, N);
            constexpr double s = DIR * sin2pi(K, N);
            v[K + N / 2] = cmul(d, cmk<C>((T)c, (T)s));
        }
        dif_level<N, K + 1, DIR, HALF>(v);
    }
}

template <int N, int DIR, bool HALF, typename C> __host__ __device__ __forceinline__ void dif(C* v) {
    if constexpr (N == 1) {
        return;
    } else if constexpr (N == 2) {
        if constexpr (HALF) v[1] = v[0];
        else rdft2<DIR>(v);
    } else if constexpr (N == 4 || N == 8) {
        if constexpr (HALF) {
#pragma unroll
            for (int i = N / 2; i < N; ++i) v[i] = cmk<C>(0, 0);
        }
        if constexpr (N == 4) rdft4<DIR>(v);
        else rdft8<DIR>(v);
    } else {
        dif_level<N, 0, DIR, HALF>(v);
        dif<N / 2, DIR, false>(v);
        dif<N / 2, DIR, false>(v + N / 2);
    }
}

}  // namespace mm
