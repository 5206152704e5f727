// Batched shared-memory FFT engine used by the demag passes.
//
// A thread block holds `nlines` complex lines of power-of-two length L in
// shared memory, element e of line b at s[e * se + b] (se = nlines + 1, the
// pad keeps strided accesses bank-conflict free).  The transform is the
// Stockham autosort formulation: stage after stage of radix R (8 while the
// remaining length allows, then 4 or 2), each taking the R elements
// j + r L/R, twiddling by w^(k r) with k = j mod Ns, doing an R-point DFT in
// registers and storing at (j / Ns) Ns R + k + r Ns, where Ns is the product
// of the radices already applied.  Output is in natural order, unnormalised.
//
// Each active thread owns 8 elements per stage (8/R groups), so a block needs
// nlines * L / 8 active threads; the stage reads all of them into registers,
// synchronises, then writes, which makes the update in place.  Extra threads
// only take part in the barriers.
#pragma once

#include "mm_internal.cuh"

namespace mm {

// multiply by DIR * i (DIR = -1 forward, +1 inverse)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
    return DIR > 0 ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

template <int DIR, typename C> __device__ __forceinline__ void dft2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2);
    C t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C* v) {
    using T = decltype(C{}.x);
    const T h = (T)0.70710678118654752440084436210484904;   // sqrt(1/2)
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    // W8^k = exp(DIR 2 pi i k / 8)
    C w1o = cmul(o1, cmk<C>(h, DIR * h));
    C w2o = mul_i<DIR>(o2);
    C w3o = cmul(o3, cmk<C>(-h, DIR * h));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1o);
    v[5] = csub(e1, w1o);
    v[2] = cadd(e2, w2o);
    v[6] = csub(e2, w2o);
    v[3] = cadd(e3, w3o);
    v[7] = csub(e3, w3o);
}

template <int R, int DIR, typename C> __device__ __forceinline__ void dftR(C* v) {
    if constexpr (R == 8) dft8<DIR>(v);
    else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
    else dft2<DIR>(v);
}

// One radix-R Stockham stage on all lines of the block.
// tw: exp(-2 pi i m / L), m < L.
template <int R, int DIR, typename C>
__device__ __forceinline__ void fft_stage(C* s, int L, int Ns, int nlines, int se, int nact,
                                          const C* __restrict__ tw) {
    constexpr int G = 8 / R;
    const int tid = threadIdx.x;
    const int per_line = L / R;
    C v[G][R];
    if (tid < nact) {
#pragma unroll
        for (int q = 0; q < G; ++q) {
            int g = q * nact + tid;
            int line = g % nlines, j = g / nlines;
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = s[(j + r * per_line) * se + line];
        }
    }
    __syncthreads();
    if (tid < nact) {
        const int step = L / (Ns * R);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            int g = q * nact + tid;
            int line = g % nlines, j = g / nlines;
            int k = j % Ns;
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw[k * r * step];
                    if (DIR > 0) w = cconj(w);
                    v[q][r] = cmul(v[q][r], w);
                }
            }
            dftR<R, DIR>(v[q]);
            int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) s[(idxD + r * Ns) * se + line] = v[q][r];
        }
    }
    __syncthreads();
}

// Full transform of every line.  Must be called by all threads of the block.
template <int DIR, typename C>
__device__ void fft_lines(C* s, int L, int nlines, int se, const C* __restrict__ tw) {
    const int nact = (nlines * L) / 8;
    int Ns = 1, rem = L;
    while (rem >= 8) {
        fft_stage<8, DIR>(s, L, Ns, nlines, se, nact, tw);
        Ns *= 8;
        rem /= 8;
    }
    if (rem == 4) fft_stage<4, DIR>(s, L, Ns, nlines, se, nact, tw);
    else if (rem == 2) fft_stage<2, DIR>(s, L, Ns, nlines, se, nact, tw);
}

}  // namespace mm
