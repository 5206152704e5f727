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

#include <type_traits>

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

// f(std::integral_constant<int, I>) for I = I0 .. N-1, unrolled at compile
// time (so twiddles indexed by I fold to constants)
template <int I, int N, typename F> __host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
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

// Complex add and subtract of float2 values as one paired FP32 instruction
// (add.rn.f32x2 / sub.rn.f32x2, sm_100 and later: each lane is rounded like
// the scalar operation, so results are unchanged and the FADD count halves).
// Other element types, and the host pass, use the scalar forms.
template <typename C> __host__ __device__ __forceinline__ C padd(C a, C b) {
#if defined(__CUDA_ARCH__)
    if constexpr (std::is_same<C, float2>::value) {
        float2 r;
        asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
            "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
        return r;
    }
#endif
    return cadd(a, b);
}
template <typename C> __host__ __device__ __forceinline__ C psub(C a, C b) {
#if defined(__CUDA_ARCH__)
    if constexpr (std::is_same<C, float2>::value) {
        float2 r;
        asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
            "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
        return r;
    }
#endif
    return csub(a, b);
}
// DIR i (a - b), formed directly in scalar: a rotated value would need its
// halves swapped before a paired instruction could use it
template <int DIR, typename C> __host__ __device__ __forceinline__ C rot_diff(C a, C b) {
    return DIR > 0 ? cmk<C>(b.y - a.y, a.x - b.x) : cmk<C>(a.y - b.y, b.x - a.x);
}

// natural-order small DFTs; ROT2 returns DIR i X[2] in place of X[2]
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft2(C* v) {
    C a = v[0], b = v[1];
    v[0] = padd(a, b);
    v[1] = psub(a, b);
}
template <int DIR, bool ROT2 = false, typename C> __host__ __device__ __forceinline__ void rdft4(C* v) {
    C t0 = padd(v[0], v[2]), t1 = psub(v[0], v[2]);
    C t2 = padd(v[1], v[3]), t3 = rot_diff<DIR>(v[1], v[3]);
    v[0] = padd(t0, t2);
    v[2] = ROT2 ? rot_diff<DIR>(t0, t2) : psub(t0, t2);
    v[1] = padd(t1, t3);
    v[3] = psub(t1, t3);
}
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft8(C* v) {
    using T = decltype(C{}.x);
    const T h = (T)0.70710678118654752440084436210484904;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    rdft4<DIR>(e);
    rdft4<DIR, true>(o);   // o[2] comes back as DIR i O[2]
    C w1o = cmk<C>(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
    C w3o = cmk<C>(-h * (o[3].x + DIR * o[3].y), h * (DIR * o[3].x - o[3].y));
    v[0] = padd(e[0], o[0]);
    v[4] = psub(e[0], o[0]);
    v[1] = padd(e[1], w1o);
    v[5] = psub(e[1], w1o);
    v[2] = padd(e[2], o[2]);
    v[6] = psub(e[2], o[2]);
    v[3] = padd(e[3], w3o);
    v[7] = psub(e[3], w3o);
}
// scalar 4- and 8-point DFTs of inputs whose upper half is zero: plain
// arithmetic, so the compiler folds the zero operands away
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft4_half(C* v) {
    const C a = v[0], b = v[1];
    const C ib = mul_dir_i(b, DIR);
    v[0] = cadd(a, b);
    v[2] = csub(a, b);
    v[1] = cadd(a, ib);
    v[3] = csub(a, ib);
}
template <int DIR, typename C> __host__ __device__ __forceinline__ void rdft8_half(C* v) {
    using T = decltype(C{}.x);
    const T h = (T)0.70710678118654752440084436210484904;
    // X[k] = E[k] + w^k O[k] with E, O the 4-point DFTs of (v0, v2) and (v1, v3)
    C e[4] = {v[0], v[2], cmk<C>(0, 0), cmk<C>(0, 0)};
    C o[4] = {v[1], v[3], cmk<C>(0, 0), cmk<C>(0, 0)};
    rdft4_half<DIR>(e);
    rdft4_half<DIR>(o);
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
        const C a = v[K];
        if constexpr (HALF) {
            if constexpr (K == 0) {
                v[K + N / 2] = a;
            } else if constexpr (4 * K == N) {
                v[K + N / 2] = mul_dir_i(a, DIR);
            } else {
                constexpr double c = cos2pi(K, N);
                constexpr double s = DIR * sin2pi(K, N);
                v[K + N / 2] = cmul(a, cmk<C>((T)c, (T)s));
            }
        } else {
            const C b = v[K + N / 2];
            v[K] = padd(a, b);
            if constexpr (K == 0) {
                v[K + N / 2] = psub(a, b);
            } else if constexpr (4 * K == N) {
                v[K + N / 2] = rot_diff<DIR>(a, b);
            } else {
                constexpr double c = cos2pi(K, N);
                constexpr double s = DIR * sin2pi(K, N);
                v[K + N / 2] = cmul(psub(a, b), cmk<C>((T)c, (T)s));
            }
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
    } else if constexpr (N == 4) {
        if constexpr (HALF) rdft4_half<DIR>(v);
        else rdft4<DIR>(v);
    } else if constexpr (N == 8) {
        if constexpr (HALF) rdft8_half<DIR>(v);
        else rdft8<DIR>(v);
    } else {
        dif_level<N, 0, DIR, HALF>(v);
        dif<N / 2, DIR, false>(v);
        dif<N / 2, DIR, false>(v + N / 2);
    }
}

}  // namespace mm
