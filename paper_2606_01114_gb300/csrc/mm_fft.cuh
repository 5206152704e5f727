// Batched shared-memory FFT engine used by the demag passes.
//
// A thread block holds `nb` batches of `NL` complex lines of power-of-two
// length L in shared memory (layout and bank swizzle: FftGeom).  The transform is the Stockham autosort
// formulation: stage after stage of radix R (8 while the remaining length
// allows, then 4 or 2), each taking the R elements j + r L/R, twiddling by
// w^(k r) with k = j mod Ns, doing an R-point DFT in registers and storing at
// (j / Ns) Ns R + k + r Ns, where Ns is the product of the radices already
// applied.  Output is in natural order, unnormalised.
//
// Pruned passes: a first stage whose inputs r >= R/2 are the zero padding
// reads and adds only the non-zero half; a last stage of which only outputs
// below L/2 are kept computes and stores only those (fft_lines HIN / HOUT).
// Every size is a power of two, so all index arithmetic is shifts and masks.
// Each active thread owns 8 elements per stage (8/R groups); a block needs
// nb * NL * L / 8 active threads.  The stage reads all of them into
// registers, synchronises, then writes, which makes the update in place.
// Extra threads only take part in the barriers.
#pragma once

#include "mm_internal.cuh"

namespace mm {

__host__ __device__ __forceinline__ int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

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
    C w1o = cmk<C>(h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x));
    C w2o = mul_i<DIR>(o2);
    C w3o = cmk<C>(-h * (o3.x + DIR * o3.y), h * (DIR * o3.x - o3.y));
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

// R-point DFT of inputs whose upper half v[R/2..R-1] is zero (not read):
// the first butterfly level becomes copies, so only the non-zero half is
// added.  Natural order out, like dftR.
template <int R, int DIR, typename C> __device__ __forceinline__ void dftR_half_in(C* v) {
    using T = decltype(C{}.x);
    if constexpr (R == 2) {
        v[1] = v[0];
    } else if constexpr (R == 4) {
        const C a = v[0], b = v[1], ib = mul_i<DIR>(v[1]);
        v[0] = cadd(a, b);
        v[2] = csub(a, b);
        v[1] = cadd(a, ib);
        v[3] = csub(a, ib);
    } else {
        // X[k] = E[k] + w^k O[k], E and O the 4-point DFTs of (v0, v2) and (v1, v3)
        const T h = (T)0.70710678118654752440084436210484904;
        C e[4] = {v[0], v[2], v[0], v[2]}, o[4] = {v[1], v[3], v[1], v[3]};
        dftR_half_in<4, DIR>(e);
        dftR_half_in<4, DIR>(o);
        const C w1o = cmk<C>(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
        const C w2o = mul_i<DIR>(o[2]);
        const C w3o = cmk<C>(-h * (o[3].x + DIR * o[3].y), h * (DIR * o[3].x - o[3].y));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1o);
        v[5] = csub(e[1], w1o);
        v[2] = cadd(e[2], w2o);
        v[6] = csub(e[2], w2o);
        v[3] = cadd(e[3], w3o);
        v[7] = csub(e[3], w3o);
    }
}

// R-point DFT keeping only the lower half of the outputs, X[0..R/2-1] in
// v[0..R/2-1] (the upper half is left undefined).
template <int R, int DIR, typename C> __device__ __forceinline__ void dftR_half_out(C* v) {
    using T = decltype(C{}.x);
    if constexpr (R == 2) {
        v[0] = cadd(v[0], v[1]);
    } else if constexpr (R == 4) {
        const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const C t2 = cadd(v[1], v[3]), t3 = mul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[1] = cadd(t1, t3);
    } else {
        const T h = (T)0.70710678118654752440084436210484904;
        C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<DIR>(e0, e1, e2, e3);
        dft4<DIR>(o0, o1, o2, o3);
        const C w1o = cmk<C>(h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x));
        const C w2o = mul_i<DIR>(o2);
        const C w3o = cmk<C>(-h * (o3.x + DIR * o3.y), h * (DIR * o3.x - o3.y));
        v[0] = cadd(e0, o0);
        v[1] = cadd(e1, w1o);
        v[2] = cadd(e2, w2o);
        v[3] = cadd(e3, w3o);
    }
}

// Geometry of the lines a block transforms (all counts powers of two except nb).
// Element e of line `line` of batch a sits at a * L * NL + swz(e) * NL + line,
// swz(e) = e ^ ((e >> 3) & sm): the XOR of the row index with bits above the
// radix-8 group spreads the rows that one warp touches in a stage (8 apart in
// the first stage) over all shared-memory banks; sm = 128 B / element size /
// NL - 1 when a 128-byte bank row holds several rows, else 0.
struct FftGeom {
    int L, lgL;     // line length
    int NL, lgNL;   // lines per batch
    int nb;         // batches
    int sm;         // row swizzle mask
    int nact;       // active threads: nb * NL * L / 8
};

__host__ __device__ inline FftGeom fft_geom(int L, int NL, int nb, int elem_bytes) {
    FftGeom g;
    g.L = L;
    g.lgL = ilog2(L);
    g.NL = NL;
    g.lgNL = ilog2(NL);
    g.nb = nb;
    int slots = 128 / elem_bytes;
    g.sm = NL < slots ? slots / NL - 1 : 0;
    g.nact = (nb * NL * L) >> 3;
    return g;
}

__device__ __forceinline__ int sidx(const FftGeom& g, int a, int e, int line) {
    return ((a << g.lgL) + (e ^ ((e >> 3) & g.sm))) * g.NL + line;
}

// twiddles w^r, r = 1..R-1, from w = tw[idx]: FP32 builds the powers by at
// most three products of the tabulated value; FP64 reads each from the table.
template <int R, int DIR, typename C>
__device__ __forceinline__ void twiddle(C* v, const C* __restrict__ tw, int k, int lgStep) {
    using T = decltype(C{}.x);
    if constexpr (sizeof(T) == 4) {
        C w1 = tw[k << lgStep];
        if (DIR > 0) w1 = cconj(w1);
        v[1] = cmul(v[1], w1);
        if constexpr (R >= 4) {
            C w2 = cmul(w1, w1);
            C w3 = cmul(w2, w1);
            v[2] = cmul(v[2], w2);
            v[3] = cmul(v[3], w3);
            if constexpr (R == 8) {
                C w4 = cmul(w2, w2);
                v[4] = cmul(v[4], w4);
                v[5] = cmul(v[5], cmul(w4, w1));
                v[6] = cmul(v[6], cmul(w3, w3));
                v[7] = cmul(v[7], cmul(w4, w3));
            }
        }
    } else {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            C w = tw[(k * r) << lgStep];
            if (DIR > 0) w = cconj(w);
            v[r] = cmul(v[r], w);
        }
    }
}

// One radix-R Stockham stage on all lines of the block.
// tw: exp(-2 pi i m / L), m < L.
// HIN (first stage only, lgNs = 0): the upper half of every line is zero,
// which in this stage is exactly the inputs r >= R/2 of each group: they are
// not read.  HOUT (last stage only, Ns = L/R): only outputs below L/2 are
// wanted, which are exactly r < R/2 of each group: the rest are neither
// computed nor stored.
template <int R, int DIR, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void fft_stage(C* s, const FftGeom& g, int lgNs, const C* __restrict__ tw) {
    constexpr int G = 8 / R;
    constexpr int lgR = R == 8 ? 3 : R == 4 ? 2 : 1;
    const int tid = threadIdx.x;
    const int lgPer = g.lgL - lgR;                 // log2(L / R)
    const int lgBatch = g.lgNL + lgPer;            // groups per batch
    const int Ns = 1 << lgNs;
    C v[G][R];
    int aa[G], ll[G], jj[G];
    if (tid < g.nact) {
#pragma unroll
        for (int q = 0; q < G; ++q) {
            int gi = q * g.nact + tid;
            int a = gi >> lgBatch;
            int rem = gi & ((1 << lgBatch) - 1);
            aa[q] = a;
            ll[q] = rem & (g.NL - 1);
            jj[q] = rem >> g.lgNL;
#pragma unroll
            for (int r = 0; r < (HIN ? R / 2 : R); ++r) v[q][r] = s[sidx(g, a, jj[q] + (r << lgPer), ll[q])];
        }
    }
    __syncthreads();
    if (tid < g.nact) {
        const int lgStep = g.lgL - lgNs - lgR;     // log2(L / (Ns R))
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int k = jj[q] & (Ns - 1);
            if (!HIN && lgNs > 0) twiddle<R, DIR>(v[q], tw, k, lgStep);
            if constexpr (HIN) dftR_half_in<R, DIR>(v[q]);
            else if constexpr (HOUT) dftR_half_out<R, DIR>(v[q]);
            else dftR<R, DIR>(v[q]);
            const int idxD = ((jj[q] >> lgNs) << (lgNs + lgR)) + k;
#pragma unroll
            for (int r = 0; r < (HOUT ? R / 2 : R); ++r) s[sidx(g, aa[q], idxD + (r << lgNs), ll[q])] = v[q][r];
        }
    }
    __syncthreads();
}

// Full transform of every line.  Must be called by all threads of the block.
// HIN: the upper half of every line is zero (the zero padding of a pruned
// forward pass); HOUT: only the lower half of the outputs is used (a pruned
// inverse pass), and the upper half of the lines is left undefined.  When
// the transform is a single stage (L <= 8) only HIN is applied.  The pruned
// first and last stages sit outside the loop of plain radix-8 stages.
template <int DIR, bool HIN = false, bool HOUT = false, typename C>
__device__ void fft_lines(C* s, const FftGeom& g, const C* __restrict__ tw) {
    int lgNs = 0, rem = g.lgL;
    if constexpr (HIN) {
        if (rem >= 3) {
            fft_stage<8, DIR, true, false>(s, g, 0, tw);
            lgNs = 3;
            rem -= 3;
        } else if (rem == 2) {
            fft_stage<4, DIR, true, false>(s, g, 0, tw);
            rem = 0;
        } else if (rem == 1) {
            fft_stage<2, DIR, true, false>(s, g, 0, tw);
            rem = 0;
        }
    }
    // bits left for the pruned last stage: its radix is 8 when lgL is a
    // multiple of 3, else 4 or 2
    const int last_bits = HOUT ? (g.lgL % 3 ? g.lgL % 3 : 3) : 0;
    while (rem >= 3 && rem > last_bits) {
        fft_stage<8, DIR>(s, g, lgNs, tw);
        lgNs += 3;
        rem -= 3;
    }
    if (rem == 0) return;
    if constexpr (HOUT) {
        if (rem == 3) fft_stage<8, DIR, false, true>(s, g, lgNs, tw);
        else if (rem == 2) fft_stage<4, DIR, false, true>(s, g, lgNs, tw);
        else fft_stage<2, DIR, false, true>(s, g, lgNs, tw);
    } else {
        if (rem == 2) fft_stage<4, DIR>(s, g, lgNs, tw);
        else fft_stage<2, DIR>(s, g, lgNs, tw);
    }
}

}  // namespace mm
