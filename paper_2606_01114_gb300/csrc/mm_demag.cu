// Demagnetisation field as a zero-padded FFT convolution (paper, Implementation
// section, Eq. 4 and the FFT paragraph after it): H = -N * M, M = Ms m,
// computed on a grid padded to P = 2n per axis (1 when n = 1), transforms
// unnormalised, inverse scaled once at the end.
//
// Five passes over HBM.  In FP32, for the common lengths, the passes are
// register-resident four-step DFTs (mm_regfft.cuh: k_xfwd_reg, k_cols_reg,
// k_zconv_reg, k_xinv_reg); otherwise, and in FP64, each is a batched
// shared-memory FFT (mm_fft.cuh).  An FP64 context in float-float mode runs
// the same generic kernels on (h + l) float pairs (mm_ff.cuh, apply_ff).
// The passes:
//   K2 x-forward: real rows of M (only the nx non-zero values are read) are
//      packed two-reals-per-complex into a length Px/2 complex FFT, then
//      unpacked to the Hx = nx + 1 non-redundant frequencies;
//   K3 y-forward: columns of Py points of which only ny are non-zero (the
//      zero half is never read);
//   K4 z-forward, the 6-component symmetric tensor product with the real
//      k-space Newell octant, and the z-inverse, fused in one pass; only the
//      nz un-padded z rows are read and written;
//   K5 y-inverse keeping ny of the Py outputs;
//   K6 x-inverse (complex-to-real by the same packing) keeping nx outputs and
//      applying the scale 1 / ((Px/2) Py Pz).
// K1 (demag_setup) computes the Newell tensor on the padded real grid in
// double-double (mm_newell.cu), runs the same passes unpruned in FP64 and
// keeps the real octant kx <= nx, ky <= Py/2, kz <= Pz/2 at path precision;
// negative frequencies follow from each component's parity.
#include <cmath>
#include <vector>

#include "mm_fft.cuh"
#include "mm_ff.cuh"
#include "mm_regfft.cuh"
#include "mm_tma.cuh"

namespace mm {
namespace {

template <typename T> using C_t = typename cx<T>::type;

// Loads and stores at the real-array boundary of the passes: S is the type
// the caller's arrays hold (m, Ms, H), T the arithmetic of the passes (the
// same type, or float-float over double arrays).
template <typename C, typename S> __device__ __forceinline__ C ld_c(const S* p, long j) {
    if constexpr (std::is_same<C, C_t<S>>::value) return reinterpret_cast<const C*>(p)[j];
    else return from_d2<C>(reinterpret_cast<const C_t<S>*>(p)[j]);
}
template <typename C, typename S> __device__ __forceinline__ void st_c(S* p, long j, C v) {
    if constexpr (std::is_same<C, C_t<S>>::value) reinterpret_cast<C*>(p)[j] = v;
    else reinterpret_cast<C_t<S>*>(p)[j] = cmk<C_t<S>>(to_d(v.x), to_d(v.y));
}
template <typename T, typename S> __device__ __forceinline__ T ld_r(S v) {
    if constexpr (std::is_same<T, S>::value) return v;
    else return from_real<T>(v);
}

// ------------------------------------------------------------------ K2
// Real rows -> packed complex FFT -> Hx frequencies.
//   B = 2^lgB rows per block, row r at in + r*in_ld, nin real values (even
//   count, rest zero); Ms: per-cell array indexed (r mod ms_rows)*in_ld + x,
//   or nullptr (scalar ms).  Complex length L = 2^lgL = Px / 2.
//   Shared memory: B lines of L (FftGeom layout); global accesses run with
//   the row index b fastest across a warp (B row segments per instruction).
// HIN: nin <= L, so the upper half of every packed line is zero padding.
template <typename T, typename S = T, bool HIN = false>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_xfwd(const S* __restrict__ in, long in_ld, int nin, const S* __restrict__ Ms, T ms,
                       long ms_rows, C_t<T>* __restrict__ out, int Hs, int lgL, long rows, int lgB,
                       const C_t<T>* __restrict__ twL, const C_t<T>* __restrict__ twP) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int L = 1 << lgL, B = 1 << lgB;
    const FftGeom g = fft_geom(L, B, 1, sizeof(C));
    const long r0 = (long)blockIdx.x << lgB;
    const int npair = nin >> 1;
    constexpr int U = 4;
    const int total = B << lgL;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = base + u * blockDim.x;
            int b = idx & (B - 1), j = idx >> lgB;
            long r = r0 + b;
            v[u] = cmk<C>(0, 0);
            if (idx < total && j < npair && r < rows) {
                v[u] = ld_c<C>(in + r * in_ld, j);
                if (Ms) {
                    C w = ld_c<C>(Ms + (r % ms_rows) * in_ld, j);
                    v[u].x *= w.x;
                    v[u].y *= w.y;
                } else {
                    v[u].x *= ms;
                    v[u].y *= ms;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = base + u * blockDim.x;
            if (idx < total) s[sidx(g, 0, idx >> lgB, idx & (B - 1))] = v[u];
        }
    }
    __syncthreads();
    fft_lines<-1, HIN>(s, g, twL);
    const T half = (T)0.5;
    // X_k = E_k - i w^k D_k, E, D the even/odd split of the packed spectrum Z
    for (int idx = threadIdx.x; idx < total + B; idx += blockDim.x) {
        int b = idx & (B - 1), k = idx >> lgB;        // k runs 0..L
        long r = r0 + b;
        if (r >= rows) continue;
        C zk = s[sidx(g, 0, k & (L - 1), b)];
        C zc = cconj(s[sidx(g, 0, (L - k) & (L - 1), b)]);
        C e = cscale(cadd(zk, zc), half);
        C d = cscale(csub(zk, zc), half);
        C wd = cmul(twP[k], d);
        out[r * Hs + k] = cmk<C>(e.x + wd.y, e.y - wd.x);
    }
}

// nx == 1: no x transform, M copied into the complex array.
template <typename T, typename S = T>
__global__ void k_x1fwd(const S* __restrict__ in, const S* __restrict__ Ms, T ms, long ms_rows,
                        C_t<T>* __restrict__ out, int Hs, long rows) {
    long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    T w = Ms ? ld_r<T>(Ms[r % ms_rows]) : ms;
    out[r * Hs] = cmk<C_t<T>>(ld_r<T>(in[r]) * w, (T)0);
}

// ------------------------------------------------------------------ K6
// Hx frequencies -> inverse packed complex FFT -> nx real outputs, scaled.
template <typename T, typename S = T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_xinv(const C_t<T>* __restrict__ in, int Hs, S* __restrict__ out, int nx, int lgL, long rows,
                       int lgB, T scale, const C_t<T>* __restrict__ twL, const C_t<T>* __restrict__ twP) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int L = 1 << lgL, B = 1 << lgB;
    const FftGeom g = fft_geom(L, B, 1, sizeof(C));
    const long r0 = (long)blockIdx.x << lgB;
    const T half = (T)0.5;
    constexpr int U = 2;
    const int total = B << lgL;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        C xk[U], xc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = base + u * blockDim.x;
            int b = idx & (B - 1), k = idx >> lgB;
            long r = r0 + b;
            xk[u] = cmk<C>(0, 0);
            xc[u] = cmk<C>(0, 0);
            if (idx < total && r < rows) {
                xk[u] = in[r * Hs + k];
                xc[u] = cconj(in[r * Hs + (L - k)]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = base + u * blockDim.x;
            if (idx >= total) continue;
            int b = idx & (B - 1), k = idx >> lgB;
            C e = cscale(cadd(xk[u], xc[u]), half);
            C o = cmul(cscale(csub(xk[u], xc[u]), half), cconj(twP[k]));   // times exp(+2 pi i k / Px)
            s[sidx(g, 0, k, b)] = cmk<C>(e.x - o.y, e.y + o.x);            // E + i O
        }
    }
    __syncthreads();
    fft_lines<+1, false, true>(s, g, twL);   // only z[j], j < nx / 2 = L / 2, is kept
    const int lgP = ilog2(nx >> 1);
    for (int idx = threadIdx.x; idx < (B << lgP); idx += blockDim.x) {
        int b = idx & (B - 1), j = idx >> lgB;
        long r = r0 + b;
        if (r >= rows) continue;
        C z = s[sidx(g, 0, j, b)];
        st_c(out + r * (long)nx, j, cmk<C>(z.x * scale, z.y * scale));
    }
}

template <typename T, typename S = T>
__global__ void k_x1inv(const C_t<T>* __restrict__ in, int Hs, S* __restrict__ out, long rows, T scale) {
    long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    out[r] = to_d(in[r * Hs].x * scale);
}

// ----------------------------------------------------------- K3 / K5
// Column FFTs along an axis with row stride `rs`: a block takes B = 2^lgB
// adjacent columns (kx) of one plane, loads nin rows (rest zero), transforms
// length L = 2^lgL, stores nout rows.  Plane p: inner index p % n_inner,
// outer p / n_inner.
// HIN: nin <= L/2 (the zero padding is the upper half); HOUT: nout <= L/2.
template <typename T, int DIR, bool HIN = false, bool HOUT = false>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_cols(const C_t<T>* in, C_t<T>* out, int lgL, int nin, int nout, int Hx, int lgB, ColGeom cg,
                       const C_t<T>* __restrict__ tw) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int L = 1 << lgL, B = 1 << lgB;
    const FftGeom g = fft_geom(L, B, 1, sizeof(C));
    const int col0 = blockIdx.x << lgB;
    const int p = blockIdx.y;
    const int pi = p % cg.n_inner, po = p / cg.n_inner;
    const C* ib = in + pi * cg.in_inner + po * cg.in_outer;
    C* ob = out + pi * cg.out_inner + po * cg.out_outer;
    constexpr int U = 4;
    const int total = L << lgB;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = base + u * blockDim.x;
            int b = idx & (B - 1), r = idx >> lgB;
            v[u] = cmk<C>(0, 0);
            if (idx < total && r < nin && col0 + b < Hx) v[u] = ib[r * cg.rs_in + col0 + b];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = base + u * blockDim.x;
            if (idx < total) s[sidx(g, 0, idx >> lgB, idx & (B - 1))] = v[u];
        }
    }
    __syncthreads();
    fft_lines<DIR, HIN, HOUT>(s, g, tw);
    for (int idx = threadIdx.x; idx < (nout << lgB); idx += blockDim.x) {
        int b = idx & (B - 1), r = idx >> lgB;
        if (col0 + b < Hx) ob[r * cg.rs_out + col0 + b] = s[sidx(g, 0, r, b)];
    }
}

// ------------------------------------------------------------------ K4
// Per (ky pair, tile of B kx): for ky and Py - ky, z-FFT of the three
// components (nz of Pz rows non-zero), H^ = -N^ M^ with the symmetric 3x3
// real tensor from the octant (N_xy odd in ky, N_xz odd in kz, N_yz odd in
// both), z-inverse, keep nz rows.  The octant rows of the tile are read once
// into shared memory and serve both ky.  Shared memory: three batches
// (components) of B lines of length Pz, then the 6 x (Pz/2+1) x B octant.
template <typename T>
__device__ __forceinline__ void zconv_one(C_t<T>* s, const T* kn, const FftGeom& g, C_t<T>* base, T sy, int nz,
                                          int lgPz, int Pz2, int lgB, int Hx, int col0, long zstride, long cstride,
                                          const C_t<T>* __restrict__ twz) {
    using C = C_t<T>;
    const int Pz = 1 << lgPz, B = 1 << lgB;
    __syncthreads();
    constexpr int U = 4;
    const int total = 3 * (Pz << lgB);
    for (int b0 = threadIdx.x; b0 < total; b0 += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = b0 + u * blockDim.x;
            int b = idx & (B - 1), rest = idx >> lgB;   // rest = c * Pz + z
            int c = rest >> lgPz, z = rest & (Pz - 1);
            v[u] = cmk<C>(0, 0);
            if (idx < total && z < nz && col0 + b < Hx) v[u] = base[c * cstride + z * zstride + b];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int idx = b0 + u * blockDim.x;
            if (idx >= total) continue;
            int b = idx & (B - 1), rest = idx >> lgB;
            s[sidx(g, rest >> lgPz, rest & (Pz - 1), b)] = v[u];
        }
    }
    __syncthreads();
    fft_lines<-1, true>(s, g, twz);          // z >= nz = Pz / 2 is the zero padding
    const int ks = Pz2 << lgB;
    for (int idx = threadIdx.x; idx < (Pz << lgB); idx += blockDim.x) {
        int b = idx & (B - 1), kz = idx >> lgB;
        int kzp = kz <= (Pz >> 1) ? kz : Pz - kz;
        T sz = kz > (Pz >> 1) ? (T)-1 : (T)1;
        const T* kk = kn + (kzp << lgB) + b;
        T nxx = kk[0], nyy = kk[ks], nzz = kk[2 * ks];
        T nxy = sy * kk[3 * ks];
        T nxz = sz * kk[4 * ks];
        T nyz = sy * sz * kk[5 * ks];
        const int o0 = sidx(g, 0, kz, b), o1 = sidx(g, 1, kz, b), o2 = sidx(g, 2, kz, b);
        C mx = s[o0], my = s[o1], mz = s[o2];
        s[o0] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
        s[o1] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
        s[o2] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
    }
    __syncthreads();
    fft_lines<+1, false, true>(s, g, twz);   // only z < nz is kept
    const int lgnz = lgPz > 0 ? lgPz - 1 : 0;               // nz = Pz / 2, or 1 when Pz = 1
    for (int idx = threadIdx.x; idx < 3 * (nz << lgB); idx += blockDim.x) {
        int b = idx & (B - 1), rest = idx >> lgB;       // rest = c * nz + z
        int c = rest >> lgnz, z = rest & (nz - 1);
        if (col0 + b < Hx) base[c * cstride + z * zstride + b] = s[sidx(g, c, z, b)];
    }
}

template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512)
    k_zconv(C_t<T>* buf, const T* __restrict__ kern, int nz, int lgPz, int Py, int Hs, int Hx, int Py2, int Pz2,
            int lgB, const C_t<T>* __restrict__ twz) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int Pz = 1 << lgPz, B = 1 << lgB;
    const FftGeom g = fft_geom(Pz, B, 3, sizeof(C));
    T* kn = reinterpret_cast<T*>(s + 3 * (Pz << lgB));     // [6][Pz2][B]
    const int col0 = blockIdx.x << lgB;
    const int kyp = blockIdx.y;                             // 0 .. Py/2
    const long zstride = (long)Py * Hs;
    const long cstride = (long)nz * zstride;
    const long kstride = (long)Pz2 * Py2 * Hs;
    for (int idx = threadIdx.x; idx < 6 * (Pz2 << lgB); idx += blockDim.x) {
        int b = idx & (B - 1), rest = idx >> lgB;           // rest = c * Pz2 + kz
        int c = rest / Pz2, kz = rest - c * Pz2;
        kn[idx] = col0 + b < Hx ? kern[c * kstride + ((long)kz * Py2 + kyp) * Hs + col0 + b] : (T)0;
    }
    zconv_one<T>(s, kn, g, buf + (long)kyp * Hs + col0, (T)1, nz, lgPz, Pz2, lgB, Hx, col0, zstride, cstride, twz);
    if (kyp != 0 && 2 * kyp != Py)
        zconv_one<T>(s, kn, g, buf + (long)(Py - kyp) * Hs + col0, (T)-1, nz, lgPz, Pz2, lgB, Hx, col0, zstride,
                     cstride, twz);
}

// ------------------------------------------------ direct DFT passes
// Transform lengths that are not powers of two (meshes such as 100 x 25)
// take these O(L^2)-per-line kernels: every output is the plain sum of its
// DFT definition, one thread per output, twiddles from the length's table
// (index (n k) mod L, advanced additively).  A correctness path beside the
// power-of-two passes, not a fast one.
inline bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Bluestein (chirp-z) passes for padded lengths P that are not powers of two
// (meshes such as 100 x 25 or 350^3): with nk = (n^2 + k^2 - (k - n)^2) / 2,
//   X[k] = sum_{n < nin} x[n] w^{nk} = a[k] sum_n (x[n] a[n]) b[k - n],
// w = exp(DIR 2 pi i / P), a[n] = exp(DIR i pi n^2 / P), b = conj(a): a
// linear convolution, done as a circular one of length M (the power of two
// >= 2P - 1, so |k - n| < P never wraps) with the power-of-two Stockham
// engine: chirp, FFT_M, times the filter spectrum (precomputed, scaled by
// 1/M), inverse FFT_M, chirp.  O(M log M) per line instead of O(nin nout).
template <typename T, int DIR>
__device__ void blue_core(C_t<T>* s, const FftGeom& g, int nin, int nout, const C_t<T>* __restrict__ chirp,
                          const C_t<T>* __restrict__ filt, const C_t<T>* __restrict__ twM) {
    using C = C_t<T>;
    const int M = g.L, B = g.NL;
    for (int idx = threadIdx.x; idx < B * nin; idx += blockDim.x) {
        const int b = idx % B, n = idx / B;
        C a = chirp[n];
        if (DIR > 0) a = cconj(a);
        const int o = sidx(g, 0, n, b);
        s[o] = cmul(s[o], a);
    }
    __syncthreads();
    fft_lines<-1>(s, g, twM);
    const C* V = filt + (DIR > 0 ? M : 0);
    for (int idx = threadIdx.x; idx < B * M; idx += blockDim.x) {
        const int b = idx % B, k = idx / B;
        const int o = sidx(g, 0, k, b);
        s[o] = cmul(s[o], V[k]);
    }
    __syncthreads();
    fft_lines<+1>(s, g, twM);
    for (int idx = threadIdx.x; idx < B * nout; idx += blockDim.x) {
        const int b = idx % B, k = idx / B;
        C a = chirp[k];
        if (DIR > 0) a = cconj(a);
        const int o = sidx(g, 0, k, b);
        s[o] = cmul(s[o], a);
    }
    __syncthreads();
}

// K3 / K5: B adjacent columns of one plane per block
template <typename T, int DIR>
__global__ void k_cols_blue(const C_t<T>* __restrict__ in, C_t<T>* __restrict__ out, int nin, int nout, int Hx,
                            int lgM, int lgB, ColGeom cg, const C_t<T>* __restrict__ chirp,
                            const C_t<T>* __restrict__ filt, const C_t<T>* __restrict__ twM) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int M = 1 << lgM, B = 1 << lgB;
    const FftGeom g = fft_geom(M, B, 1, sizeof(C));
    const int col0 = blockIdx.x << lgB;
    const int p = blockIdx.y;
    const int pi = p % cg.n_inner, po = p / cg.n_inner;
    const C* ib = in + pi * cg.in_inner + po * cg.in_outer;
    C* ob = out + pi * cg.out_inner + po * cg.out_outer;
    for (int idx = threadIdx.x; idx < B * M; idx += blockDim.x) {
        const int b = idx & (B - 1), n = idx >> lgB;
        const int col = col0 + b;
        s[sidx(g, 0, n, b)] = (n < nin && col < Hx) ? ib[(long)n * cg.rs_in + col] : cmk<C>(0, 0);
    }
    __syncthreads();
    blue_core<T, DIR>(s, g, nin, nout, chirp, filt, twM);
    for (int idx = threadIdx.x; idx < B * nout; idx += blockDim.x) {
        const int b = idx & (B - 1), k = idx >> lgB;
        const int col = col0 + b;
        if (col < Hx) ob[(long)k * cg.rs_out + col] = s[sidx(g, 0, k, b)];
    }
}

// K2: B rows per block, X_k for k < Hx of the real row (nin values, times Ms)
template <typename T>
__global__ void k_xfwd_blue(const T* __restrict__ in, long in_ld, int nin, const T* __restrict__ Ms, T ms,
                            long ms_rows, C_t<T>* __restrict__ out, int Hs, int Hx, long rows, int lgM, int lgB,
                            const C_t<T>* __restrict__ chirp, const C_t<T>* __restrict__ filt,
                            const C_t<T>* __restrict__ twM) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int M = 1 << lgM, B = 1 << lgB;
    const FftGeom g = fft_geom(M, B, 1, sizeof(C));
    const long r0 = (long)blockIdx.x << lgB;
    for (int idx = threadIdx.x; idx < B * M; idx += blockDim.x) {
        const int n = idx & (M - 1), b = idx >> lgM;
        const long r = r0 + b;
        T v = 0;
        if (n < nin && r < rows) v = in[r * in_ld + n] * (Ms ? Ms[(r % ms_rows) * in_ld + n] : ms);
        s[sidx(g, 0, n, b)] = cmk<C>(v, (T)0);
    }
    __syncthreads();
    blue_core<T, -1>(s, g, nin, Hx, chirp, filt, twM);
    for (int idx = threadIdx.x; idx < B * Hx; idx += blockDim.x) {
        const int k = idx % Hx, b = idx / Hx;
        const long r = r0 + b;
        if (r < rows) out[r * Hs + k] = s[sidx(g, 0, k, b)];
    }
}

// K6: B rows per block, out_x = scale / 2 [Re(sum_{k < nx} c_k X_k e^{+2 pi i k x / Px}) + (-1)^x Re X_nx],
// c_0 = 1, c_k = 2 (the full inverse over Px of a Hermitian spectrum)
template <typename T>
__global__ void k_xinv_blue(const C_t<T>* __restrict__ in, int Hs, T* __restrict__ out, int nx, long rows, T scale,
                            int lgM, int lgB, const C_t<T>* __restrict__ chirp, const C_t<T>* __restrict__ filt,
                            const C_t<T>* __restrict__ twM) {
    using C = C_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int M = 1 << lgM, B = 1 << lgB;
    const FftGeom g = fft_geom(M, B, 1, sizeof(C));
    const long r0 = (long)blockIdx.x << lgB;
    for (int idx = threadIdx.x; idx < B * M; idx += blockDim.x) {
        const int k = idx & (M - 1), b = idx >> lgM;
        const long r = r0 + b;
        C v = cmk<C>(0, 0);
        if (k < nx && r < rows) {
            v = in[r * Hs + k];
            if (k > 0) v = cmk<C>(v.x + v.x, v.y + v.y);
        }
        s[sidx(g, 0, k, b)] = v;
    }
    __syncthreads();
    blue_core<T, +1>(s, g, nx, nx, chirp, filt, twM);
    const T half = (T)0.5 * scale;
    for (int idx = threadIdx.x; idx < B * nx; idx += blockDim.x) {
        const int x = idx % nx, b = idx / nx;
        const long r = r0 + b;
        if (r >= rows) continue;
        const T ny_ = in[r * Hs + nx].x;
        out[r * nx + x] = half * (s[sidx(g, 0, x, b)].x + ((x & 1) ? -ny_ : ny_));
    }
}

// lines per Bluestein block: at most 1024 active threads (B M / 8) and 64 KB of shared memory
inline int blue_lines(int M, int cs) {
    int b = 1;
    while (2 * b * M / 8 <= 1024 && (size_t)2 * b * M * cs <= 65536) b *= 2;
    return b;
}

// the Bluestein arrays of an axis at precision T
template <typename T> struct BlueArrays {
    const C_t<T>* chirp;
    const C_t<T>* filt;
    const C_t<T>* tw;
};
template <typename T> BlueArrays<T> blue_arrays(const Blue& bl);
template <> BlueArrays<double> blue_arrays<double>(const Blue& bl) {
    return {(const double2*)bl.chirp, (const double2*)bl.filt, (const double2*)bl.tw};
}
template <> BlueArrays<float> blue_arrays<float>(const Blue& bl) {
    return {(const float2*)bl.chirp32, (const float2*)bl.filt32, (const float2*)bl.tw32};
}
// float-float passes need power-of-two lengths (checked when the mode is set)
template <> BlueArrays<ff> blue_arrays<ff>(const Blue&) { return {nullptr, nullptr, nullptr}; }
// Bluestein takes over from the direct DFT above this length
constexpr int kBlueMin = 64;

// K2: X_k = sum_{x < nin} M_x exp(-2 pi i k x / Px), k = 0 .. Hx - 1
template <typename T>
__global__ void k_xfwd_direct(const T* __restrict__ in, long in_ld, int nin, const T* __restrict__ Ms, T ms,
                              long ms_rows, C_t<T>* __restrict__ out, int Hs, int Hx, int Px, long rows,
                              const C_t<T>* __restrict__ twP) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * Hx) return;
    const long r = idx / Hx;
    const int k = (int)(idx % Hx);
    const T* row = in + r * in_ld;
    const T* mrow = Ms ? Ms + (r % ms_rows) * in_ld : nullptr;
    T re = 0, im = 0;
    int m = 0;
    for (int x = 0; x < nin; ++x) {
        const T v = row[x] * (mrow ? mrow[x] : ms);
        const C_t<T> w = twP[m];
        re += v * w.x;
        im += v * w.y;
        m += k;
        if (m >= Px) m -= Px;
    }
    out[r * Hs + k] = cmk<C_t<T>>(re, im);
}

// K6: out_x = scale / 2 [X_0 + (-1)^x X_nx + 2 sum_{k=1}^{nx-1} Re(X_k exp(+2 pi i k x / Px))]
// (the full inverse over Px of a Hermitian spectrum; scale = 1 / (nx Py Pz))
template <typename T>
__global__ void k_xinv_direct(const C_t<T>* __restrict__ in, int Hs, T* __restrict__ out, int nx, int Px, long rows,
                              T scale, const C_t<T>* __restrict__ twP) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * nx) return;
    const long r = idx / nx;
    const int x = (int)(idx % nx);
    const C_t<T>* row = in + r * Hs;
    T acc = 0;
    int m = x;
    for (int k = 1; k < nx; ++k) {
        const C_t<T> w = twP[m];                      // exp(-i theta); the conjugate is exp(+i theta)
        acc += row[k].x * w.x + row[k].y * w.y;       // Re(X_k conj(w))
        m += x;
        if (m >= Px) m -= Px;
    }
    const T nyq = (x & 1) ? -row[nx].x : row[nx].x;
    out[r * (long)nx + x] = (T)0.5 * scale * (row[0].x + nyq + (T)2 * acc);
}

// K3 / K5 along a strided axis: out[k] = sum_{n < nin} in[n] exp(DIR 2 pi i n k / L), k < nout
template <typename T, int DIR>
__global__ void k_cols_direct(const C_t<T>* __restrict__ in, C_t<T>* __restrict__ out, int L, int nin, int nout,
                              int Hx, ColGeom cg, const C_t<T>* __restrict__ tw) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (idx >= (long)nout * Hx) return;
    const int k = (int)(idx / Hx), col = (int)(idx % Hx);
    const int pi = p % cg.n_inner, po = p / cg.n_inner;
    const C_t<T>* ib = in + pi * cg.in_inner + po * cg.in_outer + col;
    T re = 0, im = 0;
    int m = 0;
    for (int n = 0; n < nin; ++n) {
        const C_t<T> v = ib[(long)n * cg.rs_in];
        C_t<T> w = tw[m];
        if (DIR > 0) w.y = -w.y;
        re += v.x * w.x - v.y * w.y;
        im += v.x * w.y + v.y * w.x;
        m += k;
        if (m >= L) m -= L;
    }
    out[pi * cg.out_inner + po * cg.out_outer + (long)k * cg.rs_out + col] = cmk<C_t<T>>(re, im);
}

// ------------------------------------------- FP32 register-resident passes
// K4 for Pz <= 32: one thread per (component, column) holds its whole z line
// in registers; forward DFT (upper half zero), the 3x3 product through shared
// memory (each thread forms its own component from all three), inverse DFT,
// keep the nz un-padded rows.  Block: 3 warps x 32 columns; warp c is tensor
// row c.  The block's kernel octant rows (6 components x (Pz/2 + 1) kz rows
// of 32 columns) are staged once in shared memory by 16-byte asynchronous
// copies that land while the forward DFT runs, so the product reads each
// value at a compile-time offset.  Parity signs: xy is odd in ky, xz odd in
// kz, yz odd in both (the parity of the Newell components); the kz sign is
// compile-time per row, the ky sign sy is applied once to the y spectrum and
// to row y's result.
constexpr int kZB = 32;   // columns per z-pass block

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// row C of the symmetric tensor against the staged spectra S [3][PZ][kZB]
// (the y spectrum already multiplied by sy) and kernel rows K [6][PZ/2+1][kZB]
// (storage order xx, yy, zz, xy, xz, yz); v[kz] <- -(N m)_C, row 1 divided by sy
template <int PZ, int C>
__device__ __forceinline__ void zconv_product(float2 (&v)[PZ], const float2* S, const float* K, int b) {
    constexpr int PZ2 = PZ / 2 + 1;
    constexpr int I0 = C == 0 ? 0 : C == 1 ? 3 : 4;
    constexpr int I1 = C == 0 ? 3 : C == 1 ? 1 : 5;
    constexpr int I2 = C == 0 ? 4 : C == 1 ? 5 : 2;
#pragma unroll
    for (int kz = 0; kz < PZ; ++kz) {
        const int kzp = kz <= PZ / 2 ? kz : PZ - kz;
        const bool odd = kz > PZ / 2;
        float a0 = K[(I0 * PZ2 + kzp) * kZB + b];
        float a1 = K[(I1 * PZ2 + kzp) * kZB + b];
        float a2 = K[(I2 * PZ2 + kzp) * kZB + b];
        if (odd) {
            if (C == 2) {
                a0 = -a0;
                a1 = -a1;
            } else {
                a2 = -a2;
            }
        }
        const float2 mx = S[kz * kZB + b], my = S[(PZ + kz) * kZB + b], mz = S[(2 * PZ + kz) * kZB + b];
        v[kz] = make_float2(-(a0 * mx.x + a1 * my.x + a2 * mz.x), -(a0 * mx.y + a1 * my.y + a2 * mz.y));
    }
}

// (PZ = 32: at most 80 registers, 6 blocks per SM by shared memory; at the
// compiler's own 126 registers only 5 fit, and the pass took 126 us against
// about 112 on the 512 x 512 x 16 film)
template <int PZ>
__global__ void __launch_bounds__(3 * kZB, PZ >= 32 ? 7 : 8)
    k_zconv_reg(float2* buf, const float* __restrict__ kern, int Py, int Hs, int c0, int Hx, int Py2) {
    constexpr int NZ = PZ > 1 ? PZ / 2 : 1;
    constexpr int PZ2 = PZ / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);                                // [3][PZ][kZB]
    float* K = reinterpret_cast<float*>(smem_raw + 3 * PZ * kZB * sizeof(float2));  // [6][PZ2][kZB]
    const int c = threadIdx.x / kZB, b = threadIdx.x % kZB;
    const int col0 = c0 + blockIdx.x * kZB;   // columns c0 .. Hx-1, c0 % 4 == 0
    const int col = col0 + b;
    // block rows in the order 0, Py/2, 1, Py-1, 2, Py-2, ...: the two rows that
    // share an octant row of the kernel run back to back, so its second read
    // comes from L2
    const int j = blockIdx.y;
    const int ky = j == 0 ? 0 : j == 1 ? (Py >> 1) : ((j & 1) ? Py - (j >> 1) : (j >> 1));
    const int kyp = ky <= (Py >> 1) ? ky : Py - ky;
    const bool yodd = ky > (Py >> 1);
    {
        // 16-byte chunks of the octant rows; a chunk that starts below Hx ends
        // inside the row (Hs is a multiple of 16, chunk starts of 4)
        const long kstride = (long)PZ2 * Py2 * Hs, kzs = (long)Py2 * Hs;
        const float* kb = kern + (long)kyp * Hs + col0;
        for (int q = threadIdx.x; q < 6 * PZ2 * (kZB / 4); q += 3 * kZB) {
            const int chunk = q % (kZB / 4), row = q / (kZB / 4);
            const int comp = row / PZ2, kzp = row - comp * PZ2;
            if (col0 + 4 * chunk < Hx) cp_async16(K + row * kZB + 4 * chunk, kb + comp * kstride + kzp * kzs + 4 * chunk);
        }
    }
    const bool act = col < Hx;
    const long zstride = (long)Py * Hs;
    float2* p = buf + c * (NZ * zstride) + (long)ky * Hs + col;
    float2 v[PZ];
#pragma unroll
    for (int z = 0; z < NZ; ++z) v[z] = act ? p[z * zstride] : make_float2(0.f, 0.f);
    dif<PZ, -1, (PZ > 1)>(v);
    if (c == 1 && yodd) {
#pragma unroll
        for (int kz = 0; kz < PZ; ++kz) v[kz] = make_float2(-v[kz].x, -v[kz].y);
    }
#pragma unroll
    for (int kz = 0; kz < PZ; ++kz) S[(c * PZ + kz) * kZB + b] = v[dif_pos<PZ>(kz)];
    cp_async_wait_all();
    __syncthreads();
    if (c == 0) zconv_product<PZ, 0>(v, S, K, b);
    else if (c == 1) zconv_product<PZ, 1>(v, S, K, b);
    else zconv_product<PZ, 2>(v, S, K, b);
    dif<PZ, +1, false>(v);
    if (act) {
        const float sg = (c == 1 && yodd) ? -1.f : 1.f;
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            const float2 o = v[dif_pos<PZ>(z)];
            p[z * zstride] = make_float2(sg * o.x, sg * o.y);
        }
    }
}

// K6 for the packed complex length L = L1 x L2 (64 <= L <= 256, L1 >= L2;
// L = 512 takes k_xinv_pk): four-step transform of B rows through shared
// memory, with the complex-to-real packing as a further shared-memory pass
// before it.
// Level-1 threads (t < L2) hold z[t + L2 n1]; level-2 threads (k1 < L1)
// hold row k1 of the L1 x L2 transpose, XOR-swizzled (xsw, shared with K2).
template <int L1, int L2> __device__ __forceinline__ int xsw(int k1, int n2) {
    return k1 * L2 + (n2 ^ (k1 & (L2 - 1) & 15));
}

template <int L1, int L2>
__global__ void __launch_bounds__(128, (L1 * L2 >= 512) ? 6 : 8)
    k_xinv_reg(const float2* __restrict__ in, int Hs, float* __restrict__ out, long rows, float scale,
               const float2* __restrict__ twL, const float2* __restrict__ twP) {
    constexpr int L = L1 * L2, B = 4, NX = L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);      // [B][L]
    const int tid = threadIdx.x;
    const long r0 = (long)blockIdx.x * B;
    constexpr int U = 4;
    static_assert(L2 % U == 0, "the row tile must split evenly over the unrolled loads");
    for (int base = tid; base < B * L; base += U * blockDim.x) {
        float2 xk[U], xc[U], w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            const int b = idx / L, k = idx % L;
            const long r = r0 + b;
            const bool ok = r < rows;
            xk[u] = ok ? in[r * Hs + k] : make_float2(0.f, 0.f);
            xc[u] = ok ? in[r * Hs + (L - k)] : make_float2(0.f, 0.f);
            w[u] = twP[k];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            const float2 c = cconj(xc[u]);
            const float2 e = cscale(cadd(xk[u], c), 0.5f);
            const float2 o = cmul(cscale(csub(xk[u], c), 0.5f), cconj(w[u]));   // times exp(+2 pi i k / Px)
            S[idx] = make_float2(e.x - o.y, e.y + o.x);                         // E + i O
        }
    }
    __syncthreads();
    float2 v[L1];
    const int t = tid % L2, b1 = tid / L2;
    const bool lvl1 = tid < B * L2;
    if (lvl1) {
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) v[n1] = S[b1 * L + t + L2 * n1];
        dif<L1, +1, false>(v);
    }
    __syncthreads();
    if (lvl1) {
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 y = v[dif_pos<L1>(k1)];
            if (k1 > 0) y = cmul(y, cconj(twL[t * k1]));
            S[b1 * L + xsw<L1, L2>(k1, t)] = y;
        }
    }
    __syncthreads();
    const int k1 = tid % L1, b2 = tid / L1;
    const long r = r0 + b2;
    float2 u[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) u[n2] = S[b2 * L + xsw<L1, L2>(k1, n2)];
    dif<L2, +1, false>(u);
    if (r < rows) {
        float2* op = reinterpret_cast<float2*>(out + r * NX);
#pragma unroll
        for (int k2 = 0; k2 < L2 / 2; ++k2) {
            const float2 z = u[dif_pos<L2>(k2)];
            op[k1 + L1 * k2] = make_float2(z.x * scale, z.y * scale);
        }
    }
}

// K6 for L = 512 as 16 x 32: level 1 with L2 = 32 threads per row (all 128
// threads of the block) forms the packed values in its loads (X[n] and
// X[L - n] straight from the spectrum, the twiddle exp(+2 pi i n / Px) as a
// per-thread part times a compile-time part), so the packing needs no
// shared-memory pass; one shared-memory transpose; level 2 on B x L1
// threads.  (The same packing with the 32 x 16 split, where only half the
// threads load, was 2 % slower than k_xinv_reg.)
template <int L1, int L2>
__global__ void __launch_bounds__(128, 6)
    k_xinv_pk(const float2* __restrict__ in, int Hs, float* __restrict__ out, long rows, float scale,
              const float2* __restrict__ twL, const float2* __restrict__ twP) {
    constexpr int L = L1 * L2, B = 4, NX = L;
    static_assert(B * L2 == 128, "level 1 takes every thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);      // [B][L]
    const int tid = threadIdx.x;
    const long r0 = (long)blockIdx.x * B;
    {
        const int t = tid % L2, b1 = tid / L2;
        const long r = r0 + b1;
        const bool ok = r < rows;
        const float2* irow = in + (ok ? r : 0) * Hs;
        const float2 wt = cconj(twP[t]);
        float2 v[L1];
        static_for<0, L1>([&](auto N1) {
            constexpr int n1 = decltype(N1)::value;
            const int n = t + L2 * n1;
            const float2 xk = ok ? irow[n] : make_float2(0.f, 0.f);
            const float2 xc = ok ? irow[L - n] : make_float2(0.f, 0.f);
            const float2 c = cconj(xc);
            const float2 e = cscale(cadd(xk, c), 0.5f);
            float2 o = cmul(cscale(csub(xk, c), 0.5f), wt);
            if constexpr (n1 > 0) {
                constexpr double cc = cos2pi(n1, 2 * L1), ss = sin2pi(n1, 2 * L1);
                o = cmul(o, make_float2((float)cc, (float)ss));
            }
            v[n1] = make_float2(e.x - o.y, e.y + o.x);
        });
        dif<L1, +1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 y = v[dif_pos<L1>(k1)];
            if (k1 > 0) y = cmul(y, cconj(twL[t * k1]));
            S[b1 * L + xsw<L1, L2>(k1, t)] = y;
        }
    }
    __syncthreads();
    if (tid < B * L1) {
        const int k1 = tid % L1, b2 = tid / L1;
        const long r = r0 + b2;
        float2 u[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) u[n2] = S[b2 * L + xsw<L1, L2>(k1, n2)];
        dif<L2, +1, false>(u);
        if (r < rows) {
            float2* op = reinterpret_cast<float2*>(out + r * NX);
#pragma unroll
            for (int k2 = 0; k2 < L2 / 2; ++k2) {
                const float2 z = u[dif_pos<L2>(k2)];
                op[k1 + L1 * k2] = make_float2(z.x * scale, z.y * scale);
            }
        }
    }
}

// K2 for the packed complex length L = L1 x L2 (64 <= L <= 512, L1 >= L2):
// four-step transform of B rows, level 1 through shared memory, with the
// real-to-complex unpacking done in registers: after level 2,
// thread (k1, b) holds Z[k1 + L1 k2] of its row, and the partner value
// conj Z[L - k] comes from lane L1 - k1 of the same row by a warp shuffle
// (lane 0 of the row pairs with itself, k2 <-> L2 - k2).  The twiddle w^k,
// w = exp(-2 pi i / Px), splits into a per-thread w^k1 (one table read) and
// a compile-time w^(L1 k2).  Each output row is written straight from
// registers: no shared-memory round trip and no barrier after level 2.
// PQ (L = 512): level 1 runs on all 128 threads instead of B L2 = 64, each
// thread taking one output parity of the L1-point transform (16 values
// instead of 32), so no warp idles at the barrier.
template <int L1, int L2, bool PQ = false>
__global__ void __launch_bounds__(128, 7)
    k_xfwd_reg(const float* __restrict__ in, const float* __restrict__ Ms, float ms, long ms_rows,
                float2* __restrict__ out, int Hs, long rows, const float2* __restrict__ twL,
                const float2* __restrict__ twP) {
    constexpr int L = L1 * L2, B = 4, NX = L;
    static_assert(32 % L1 == 0 || L1 % 32 == 0, "rows must not straddle warps unevenly");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);      // [B][L]
    const int tid = threadIdx.x;
    const long r0 = (long)blockIdx.x * B;
    if constexpr (PQ) {
        // level 1 on every thread: the L1-point transform of L1/2 non-zero
        // inputs split by output parity q (warps 0-1 even k1, 2-3 odd k1):
        // X[2j] = DFT_{L1/2}(x)[j], X[2j + 1] = DFT_{L1/2}(x w^n)[j]
        static_assert(2 * B * L2 == B * L1, "two parity classes fill the block");
        constexpr int H = L1 / 2;
        const int t = tid % L2, b = (tid / L2) % B, q = tid / (L2 * B);
        const long r = r0 + b;
        const bool act = r < rows;
        const float2* rowp = reinterpret_cast<const float2*>(in + (act ? r : 0) * NX);
        const float2* msp = Ms ? reinterpret_cast<const float2*>(Ms + ((act ? r : 0) % ms_rows) * NX) : nullptr;
        float2 v[H];
#pragma unroll
        for (int n1 = 0; n1 < H; ++n1) {
            const int j = t + L2 * n1;
            float2 a = act ? rowp[j] : make_float2(0.f, 0.f);
            if (msp) {
                float2 w = msp[j];
                a.x *= w.x;
                a.y *= w.y;
            } else {
                a.x *= ms;
                a.y *= ms;
            }
            v[n1] = a;
        }
        if (q) {
            static_for<1, H>([&](auto N) {
                constexpr int n = decltype(N)::value;
                constexpr double c = cos2pi(n, L1), sn = -sin2pi(n, L1);
                v[n] = cmul(v[n], make_float2((float)c, (float)sn));
            });
        }
        dif<H, -1, false>(v);
#pragma unroll
        for (int jj = 0; jj < H; ++jj) {
            const int k1 = 2 * jj + q;
            float2 y = v[dif_pos<H>(jj)];
            if (k1 > 0) y = cmul(y, twL[t * k1]);
            S[b * L + xsw<L1, L2>(k1, t)] = y;
        }
    } else if (tid < B * L2) {
        const int t = tid % L2, b = tid / L2;
        const long r = r0 + b;
        const bool act = r < rows;
        const float2* rowp = reinterpret_cast<const float2*>(in + (act ? r : 0) * NX);
        const float2* msp = Ms ? reinterpret_cast<const float2*>(Ms + ((act ? r : 0) % ms_rows) * NX) : nullptr;
        float2 v[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1 / 2; ++n1) {
            const int j = t + L2 * n1;
            float2 a = act ? rowp[j] : make_float2(0.f, 0.f);
            if (msp) {
                float2 w = msp[j];
                a.x *= w.x;
                a.y *= w.y;
            } else {
                a.x *= ms;
                a.y *= ms;
            }
            v[n1] = a;
        }
        dif<L1, -1, true>(v);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 y = v[dif_pos<L1>(k1)];
            if (k1 > 0) y = cmul(y, twL[t * k1]);
            S[b * L + xsw<L1, L2>(k1, t)] = y;
        }
    }
    __syncthreads();
    const int k1 = tid % L1, b2 = tid / L1;
    float2 u[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) u[n2] = S[b2 * L + xsw<L1, L2>(k1, n2)];
    dif<L2, -1, false>(u);
    const int lane = tid & 31;
    const int partner = lane - k1 + ((L1 - k1) & (L1 - 1));
    const long r = r0 + b2;
    const float2 wk1 = twP[k1];
    float2* orow = out + (r < rows ? r : 0) * Hs;
    static_for<0, L2>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        const float2 zk = u[dif_pos<L2>(k2)];
        const float2 zs = u[dif_pos<L2>(L2 - 1 - k2)];
        float2 zp;
        zp.x = __shfl_sync(0xffffffffu, zs.x, partner);
        zp.y = __shfl_sync(0xffffffffu, zs.y, partner);
        if (k1 == 0) zp = u[dif_pos<L2>((L2 - k2) & (L2 - 1))];
        const float2 zc = cconj(zp);
        const float2 e = cscale(cadd(zk, zc), 0.5f);
        float2 d = cscale(csub(zk, zc), 0.5f);
        if constexpr (k2 > 0) {
            constexpr double c = cos2pi(k2, 2 * L2), sn = -sin2pi(k2, 2 * L2);
            d = cmul(d, make_float2((float)c, (float)sn));
        }
        const float2 wd = cmul(wk1, d);
        if (r < rows) orow[k1 + L1 * k2] = make_float2(e.x + wd.y, e.y - wd.x);
        if constexpr (k2 == 0) {
            if (k1 == 0 && r < rows) orow[L] = make_float2(zk.x - zk.y, 0.f);
        }
    });
}

// K6 for L = 512 (nx = 512), TMA-fed: the arithmetic of k_xinv_pk<16, 32>,
// with tiles of kXB spectrum rows (Hs = 528, 16.5 KB, contiguous) streamed
// into shared memory by one 1-D bulk copy each, a 2-stage mbarrier ring per
// persistent block, and the level-1 transpose written in place over the
// stage's input.  Per tile: wait; level-1 loads from the stage with the
// complex-to-real packing; barrier (past it, every thread has finished the
// previous tile, so thread 0 re-arms that tile's stage with the next tile);
// level-1 DFT and transpose into the stage; barrier; level 2 and the global
// stores, which overlap the copy in flight.  Bounded waits as in k_cols_tma.
// (The same ring for K2 ran 37.0 us against 33.5 us for k_xfwd_reg: that
// pass keeps its direct loads.)
constexpr int kXB = 4;        // rows per tile
constexpr int kXHs = 528;     // spectrum row stride for nx = 512
constexpr long kTmaWaitLimit = 1L << 24;   // polls of a TMA-fed pass's mbarrier before it gives up

__global__ void __launch_bounds__(128, 6)
    k_xinv_tma(const float2* __restrict__ in, float* __restrict__ out, long rows, int ntiles, float scale,
               const float2* __restrict__ twL, const float2* __restrict__ twP, int* __restrict__ status) {
    constexpr int L1 = 16, L2 = 32, L = L1 * L2, B = kXB, NX = L, S = 2, HS = kXHs;
    constexpr int STAGE = B * HS;                  // float2 per stage (>= B L)
    static_assert(B * HS >= B * L && (B * HS * 8) % 128 == 0, "stage holds the input tile and the transpose");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((128u - (tma::smem_addr(smem_raw) & 127u)) & 127u);
    float2* st = reinterpret_cast<float2*>(sm);                                    // [S][B][HS]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)S * STAGE * sizeof(float2));
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < S; ++q) tc5::mbar_init(tma::smem_addr(&bar[q]), 1);
        tma::fence_init();
    }
    __syncthreads();
    auto issue = [&](int tile, int q) {
        const long r0 = (long)tile * B;
        const long nr = rows - r0 < B ? rows - r0 : B;
        const uint32_t bytes = (uint32_t)(nr * HS * sizeof(float2));
        const uint32_t mb = tma::smem_addr(&bar[q]);
        tma::expect_tx(mb, bytes);
        tma::load_1d(tma::smem_addr(st + (size_t)q * STAGE), in + r0 * HS, bytes, mb);
    };
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            const int tile = blockIdx.x + q * gridDim.x;
            if (tile < ntiles) issue(tile, q);
        }
    }
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int sidx_ = i % S;
        float2* Sb = st + (size_t)sidx_ * STAGE;
        const long r0 = (long)tile * B;
        const bool ok = tc5::mbar_wait(tma::smem_addr(&bar[sidx_]), (uint32_t)((i / S) & 1), kTmaWaitLimit);
        // level 1 with the packing folded into the loads (as k_xinv_pk)
        const int t = tid % L2, b1 = tid / L2;
        const bool act = r0 + b1 < rows;
        const float2* irow = Sb + b1 * HS;
        const float2 wt = cconj(twP[t]);
        float2 v[L1];
        static_for<0, L1>([&](auto N1) {
            constexpr int n1 = decltype(N1)::value;
            const int n = t + L2 * n1;
            const float2 xk = act ? irow[n] : make_float2(0.f, 0.f);
            const float2 xc = act ? irow[L - n] : make_float2(0.f, 0.f);
            const float2 c = cconj(xc);
            const float2 e = cscale(cadd(xk, c), 0.5f);
            float2 o = cmul(cscale(csub(xk, c), 0.5f), wt);
            if constexpr (n1 > 0) {
                constexpr double cc = cos2pi(n1, 2 * L1), ss = sin2pi(n1, 2 * L1);
                o = cmul(o, make_float2((float)cc, (float)ss));
            }
            v[n1] = make_float2(e.x - o.y, e.y + o.x);
        });
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(status, 0, (int)MM_ERR_TIMEOUT);
                for (int j = i; j < i + S; ++j) {
                    if (blockIdx.x + j * gridDim.x < ntiles)
                        tc5::mbar_wait(tma::smem_addr(&bar[j % S]), (uint32_t)((j / S) & 1), kTmaWaitLimit);
                }
            }
            return;
        }
        // every thread is past the previous tile, whose stage now takes tile i + 1
        if (tid == 0 && i > 0) {
            const int nt = tile + gridDim.x;
            if (nt < ntiles) {
                tma::fence_async();
                issue(nt, (i + 1) % S);
            }
        }
        dif<L1, +1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 y = v[dif_pos<L1>(k1)];
            if (k1 > 0) y = cmul(y, cconj(twL[t * k1]));
            Sb[b1 * L + xsw<L1, L2>(k1, t)] = y;
        }
        __syncthreads();
        if (tid < B * L1) {
            const int k1 = tid % L1, b2 = tid / L1;
            float2 u[L2];
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) u[n2] = Sb[b2 * L + xsw<L1, L2>(k1, n2)];
            dif<L2, +1, false>(u);
            const long r = r0 + b2;
            if (r < rows) {
                float2* op = reinterpret_cast<float2*>(out + r * NX);
#pragma unroll
                for (int k2 = 0; k2 < L2 / 2; ++k2) {
                    const float2 z = u[dif_pos<L2>(k2)];
                    op[k1 + L1 * k2] = make_float2(z.x * scale, z.y * scale);
                }
            }
        }
    }
}

// K3 / K5 for L = L1 x L2 (64 <= L <= 1024): four-step transform of B
// columns.  Level 1: thread t < L2 of a column holds x[t + L2 n1], n1 < L1,
// (upper half zero when PIN), DFT over n1, twiddle w_L^(t k1), store to
// shared memory.  Level 2: thread k1 < L1 holds the L2 values of its row,
// DFT over n2, X[k1 + L1 k2] (only k2 < L2/2 when POUT).  Shared rows are
// XOR-swizzled so both levels hit distinct banks.
template <int L1, int L2, int DIR, bool PIN, bool POUT>
__global__ void __launch_bounds__(256)
    k_cols_reg(const float2* in, float2* out, int c0, int Hx, int lgB, ColGeom cg, const float2* __restrict__ tw) {
    constexpr int L = L1 * L2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);      // [L1][L2][B]
    const int B = 1 << lgB;
    const int m = B < 16 ? (16 >> lgB) - 1 : 0;
    const int b = threadIdx.x & (B - 1), t = threadIdx.x >> lgB;
    const int col = c0 + (blockIdx.x << lgB) + b;   // columns c0 .. Hx-1
    const bool act = col < Hx;
    const int p = blockIdx.y;
    const int pi = p % cg.n_inner, po = p / cg.n_inner;
    const float2* ib = in + pi * cg.in_inner + po * cg.in_outer + (act ? col : 0);
    float2* ob = out + pi * cg.out_inner + po * cg.out_outer + col;
    if (t < L2) {
        float2 v[L1];
        constexpr int NIN = PIN ? L1 / 2 : L1;
#pragma unroll
        for (int n1 = 0; n1 < NIN; ++n1) v[n1] = act ? ib[(long)(t + L2 * n1) * cg.rs_in] : make_float2(0.f, 0.f);
        dif<L1, DIR, PIN>(v);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 y = v[dif_pos<L1>(k1)];
            if (k1 > 0) {
                float2 w = tw[t * k1];
                if (DIR > 0) w.y = -w.y;
                y = cmul(y, w);
            }
            S[((k1 * L2) + (t ^ (k1 & m))) * B + b] = y;
        }
    }
    __syncthreads();
    if (t < L1) {
        float2 u[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) u[n2] = S[((t * L2) + (n2 ^ (t & m))) * B + b];
        dif<L2, DIR, false>(u);
        constexpr int NOUT = POUT ? L2 / 2 : L2;
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < NOUT; ++k2) ob[(long)(t + L1 * k2) * cg.rs_out] = u[dif_pos<L2>(k2)];
        }
    }
}

// K3 / K5, TMA-fed (Py = L = 512 or 1024, the pruning of the product path):
// the same four-step arithmetic as k_cols_reg, with the column tiles
// streamed into shared memory by the copy engine.  A persistent block (one
// per SM: two 64 KB stages at L = 1024) walks tiles of kYB columns of one
// plane, tile = cx + ntx p.  Per tile:
//   wait for its stage's mbarrier (the tile's nin rows, in boxes of 256
//   rows x kYB columns, row-major [row][b]);
//   level 1 reads its inputs from the stage; barrier; writes its twiddled
//   outputs back into the same stage buffer (the transpose, XOR-swizzled
//   as in k_cols_reg); barrier; level 2 reads them; barrier;
//   thread 0 re-arms the stage and issues the copies of tile + 2 grid;
//   level 2's DFT and its global stores overlap that copy and the one
//   already in flight into the other stage.
// The register passes leave DRAM idle while a block computes and have two
// blocks per SM to cover it; here the next tile is always landing.
// Waits are bounded: a wait that gives up raises TIMEOUT in the device
// status, waits (bounded) for the copies still in flight and returns.
constexpr int kYB = 8;          // columns per tile (64-byte rows)
constexpr int kYStages = 2;

template <int L1, int L2, int DIR, bool PIN, bool POUT>
__global__ void __launch_bounds__(kYB * (L1 > L2 ? L1 : L2), L1 * L2 >= 1024 ? 1 : 2)
    k_cols_tma(const __grid_constant__ CUtensorMap tin, float2* __restrict__ out, int Hx, int ntx, int ntiles,
               long rs_out, long out_plane, const float2* __restrict__ tw, int* __restrict__ status) {
    constexpr int L = L1 * L2, B = kYB, S = kYStages;
    constexpr int NIN = PIN ? L / 2 : L;
    constexpr int BOX = NIN < 256 ? NIN : 256;
    constexpr int NBOX = NIN / BOX;
    constexpr uint32_t TX = (uint32_t)NIN * B * sizeof(float2);
    constexpr int m = (16 / B) - 1;
    static_assert(NIN % BOX == 0, "the rows split into whole boxes");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // copy destinations 128-byte aligned (the launch adds 128 bytes of slack)
    unsigned char* sm = smem_raw + ((128u - (tma::smem_addr(smem_raw) & 127u)) & 127u);
    float2* st = reinterpret_cast<float2*>(sm);                                    // [S][L][B]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)S * L * B * sizeof(float2));
    const int tid = threadIdx.x;
    const int b = tid % B, t = tid / B;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) tc5::mbar_init(tma::smem_addr(&bar[s]), 1);
        tma::fence_init();
    }
    __syncthreads();
    auto issue = [&](int tile, int s) {
        const int cx = tile % ntx, p = tile / ntx;
        const uint32_t mb = tma::smem_addr(&bar[s]);
        tma::expect_tx(mb, TX);
#pragma unroll
        for (int q = 0; q < NBOX; ++q)
            tma::load_3d(tma::smem_addr(st + ((size_t)s * L + q * BOX) * B), &tin, 2 * B * cx, q * BOX, p, mb);
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            const int tile = blockIdx.x + s * gridDim.x;
            if (tile < ntiles) issue(tile, s);
        }
    }
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int s = i % S;
        float2* Sb = st + (size_t)s * L * B;
        const bool ok = tc5::mbar_wait(tma::smem_addr(&bar[s]), (uint32_t)((i / S) & 1), kTmaWaitLimit);
        float2 v[L1];
        if (t < L2) {
            constexpr int NI = PIN ? L1 / 2 : L1;
#pragma unroll
            for (int n1 = 0; n1 < NI; ++n1) v[n1] = Sb[(t + L2 * n1) * B + b];
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(status, 0, (int)MM_ERR_TIMEOUT);
                for (int j = i; j < i + S; ++j) {
                    if (blockIdx.x + j * gridDim.x < ntiles)
                        tc5::mbar_wait(tma::smem_addr(&bar[j % S]), (uint32_t)((j / S) & 1), kTmaWaitLimit);
                }
            }
            return;
        }
        if (t < L2) {
            dif<L1, DIR, PIN>(v);
#pragma unroll
            for (int k1 = 0; k1 < L1; ++k1) {
                float2 y = v[dif_pos<L1>(k1)];
                if (k1 > 0) {
                    float2 w = tw[t * k1];
                    if (DIR > 0) w.y = -w.y;
                    y = cmul(y, w);
                }
                Sb[((k1 * L2) + (t ^ (k1 & m))) * B + b] = y;
            }
        }
        __syncthreads();
        float2 u[L2];
        if (t < L1) {
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) u[n2] = Sb[((t * L2) + (n2 ^ (t & m))) * B + b];
        }
        __syncthreads();
        if (tid == 0) {
            const int nt = tile + S * gridDim.x;
            if (nt < ntiles) {
                tma::fence_async();
                issue(nt, s);
            }
        }
        if (t < L1) {
            dif<L2, DIR, false>(u);
            const int cx = tile % ntx, p = tile / ntx;
            const int col = cx * B + b;
            constexpr int NOUT = POUT ? L2 / 2 : L2;
            if (col < Hx) {
                float2* ob = out + (long)p * out_plane + col;
#pragma unroll
                for (int k2 = 0; k2 < NOUT; ++k2) ob[(long)(t + L1 * k2) * rs_out] = u[dif_pos<L2>(k2)];
            }
        }
    }
}

// K1 tail: keep the real octant of the transformed component, at precision T.
template <typename T>
__global__ void k_extract(const double2* __restrict__ X, int Py, int Hs, int Hx, int Py2, int Pz2,
                          T* __restrict__ kern) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)Pz2 * Py2 * Hs;
    if (idx >= total) return;
    int kx = (int)(idx % Hs);
    int ky = (int)((idx / Hs) % Py2);
    int kz = (int)(idx / ((long)Hs * Py2));
    T v = 0;
    if (kx < Hx) v = (T)X[((long)kz * Py + ky) * Hs + kx].x;
    kern[idx] = v;
}

// ------------------------------------------------------------ launch helpers
inline int block_threads(int nact) {
    int t = nact < 64 ? 64 : nact;
    t = (t + 31) / 32 * 32;
    return t > 1024 ? 1024 : t;
}

inline int clamp_pow2(int v, int lo, int hi) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    if (p < lo) p = lo;
    if (p > hi) p = hi;
    return p;
}

// rows per block of the x passes: about 256 active threads, at least 4 rows
inline int x_rows_per_block(int L) { return clamp_pow2(2048 / L, 4, 64); }
// columns per block of the y passes: at least 32 bytes of each row, at most
// 512 active threads
inline int col_tile(int L, int cs) { return clamp_pow2(4096 / L, 32 / cs, 32); }
// columns per block of the z pass (three components each): at most 1024
// (FP32) or 512 (FP64) active threads, at least 32 bytes of each row where
// that limit allows
inline int z_tile(int Pz, int cs) {
    int cap = (cs == 8 ? 8192 : 4096) / (3 * Pz);       // nact = 3 B Pz / 8 <= 1024 or 512
    int lo = 32 / cs;
    int b = Pz >= 8 ? 1024 / Pz : 32;
    if (b > cap) b = cap;
    if (b < lo && lo <= cap) b = lo;
    b = clamp_pow2(b, 1, 32);
    if (Pz < 8 && b * Pz < 8) b = 8 / Pz;
    return b;
}

template <typename T> const C_t<T>* table(const mm_ctx* ctx, long off);
template <> const double2* table<double>(const mm_ctx* ctx, long off) { return (const double2*)ctx->tw.f64 + off; }
template <> const float2* table<float>(const mm_ctx* ctx, long off) { return (const float2*)ctx->tw.f32 + off; }

int set_smem(mm_ctx* ctx, const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) {
        MM_CUDA_CHECK(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    }
    return MM_OK;
}

template <int L1, int L2>
int launch_xfwd_reg(mm_ctx* ctx, const float* in, const float* Ms, float ms, long ms_rows, float2* out, long rows,
                    const float2* twL, const float2* twP) {
    constexpr int B = 4;
    const size_t smem = (size_t)B * L1 * L2 * sizeof(float2);
    if constexpr (L1 == 32 && L2 == 16) {
        // level 1 split by output parity over all 128 threads: 39.0 -> 33.4 us on the 512 x 512 x 16 film
        int rc = set_smem(ctx, (const void*)k_xfwd_reg<L1, L2, true>, smem);
        if (rc) return rc;
        k_xfwd_reg<L1, L2, true><<<(unsigned)((rows + B - 1) / B), B * L1, smem, ctx->stream>>>(
            in, Ms, ms, ms_rows, out, ctx->Hs, rows, twL, twP);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    int rc = set_smem(ctx, (const void*)k_xfwd_reg<L1, L2>, smem);
    if (rc) return rc;
    k_xfwd_reg<L1, L2><<<(unsigned)((rows + B - 1) / B), B * L1, smem, ctx->stream>>>(in, Ms, ms, ms_rows, out,
                                                                                   ctx->Hs, rows, twL, twP);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int try_xfwd_reg(mm_ctx* ctx, const float* in, const float* Ms, float ms, long ms_rows, float2* out, long rows,
                 const float2* twL, const float2* twP, int L, bool* done) {
    *done = true;
    switch (L) {
        case 64: return launch_xfwd_reg<8, 8>(ctx, in, Ms, ms, ms_rows, out, rows, twL, twP);
        case 128: return launch_xfwd_reg<16, 8>(ctx, in, Ms, ms, ms_rows, out, rows, twL, twP);
        case 256: return launch_xfwd_reg<16, 16>(ctx, in, Ms, ms, ms_rows, out, rows, twL, twP);
        case 512: return launch_xfwd_reg<32, 16>(ctx, in, Ms, ms, ms_rows, out, rows, twL, twP);
        default: *done = false; return MM_OK;
    }
}
template <typename T>
int try_xfwd_reg(mm_ctx*, const T*, const T*, T, long, C_t<T>*, long, const C_t<T>*, const C_t<T>*, int, bool* done) {
    *done = false;
    return MM_OK;
}

template <int L1, int L2>
int launch_xinv_reg(mm_ctx* ctx, const float2* in, float* out, long rows, float scale, const float2* twL,
                    const float2* twP) {
    constexpr int B = 4;
    const size_t smem = (size_t)B * L1 * L2 * sizeof(float2);
    if constexpr (L1 * L2 == 512) {
        // 16 x 32 with the packing folded into the level-1 loads: 53.3 -> 35.5 us on the 512 x 512 x 16 film
        int rc = set_smem(ctx, (const void*)k_xinv_pk<16, 32>, smem);
        if (rc) return rc;
        k_xinv_pk<16, 32><<<(unsigned)((rows + B - 1) / B), 128, smem, ctx->stream>>>(in, ctx->Hs, out, rows, scale,
                                                                                     twL, twP);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    int rc = set_smem(ctx, (const void*)k_xinv_reg<L1, L2>, smem);
    if (rc) return rc;
    k_xinv_reg<L1, L2><<<(unsigned)((rows + B - 1) / B), B * L1, smem, ctx->stream>>>(in, ctx->Hs, out, rows, scale,
                                                                                   twL, twP);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int try_xinv_reg(mm_ctx* ctx, const float2* in, float* out, long rows, float scale, const float2* twL,
                 const float2* twP, int L, bool* done) {
    *done = true;
    switch (L) {
        case 64: return launch_xinv_reg<8, 8>(ctx, in, out, rows, scale, twL, twP);
        case 128: return launch_xinv_reg<16, 8>(ctx, in, out, rows, scale, twL, twP);
        case 256: return launch_xinv_reg<16, 16>(ctx, in, out, rows, scale, twL, twP);
        case 512: return launch_xinv_reg<32, 16>(ctx, in, out, rows, scale, twL, twP);
        default: *done = false; return MM_OK;
    }
}

// TMA-fed x inverse (FP32, nx = 512): shared memory per block, and the
// persistent grid (SMs x resident blocks), found once per context
constexpr size_t kXinvTmaSmem = 2 * (size_t)kXB * kXHs * sizeof(float2) + 2 * sizeof(uint64_t) + 128;

void xtma_prepare(mm_ctx* ctx) {
    ctx->xtma_state = -1;
    int nsm = 0, per = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_xinv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kXinvTmaSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_xinv_tma, 128, kXinvTmaSmem) !=
            cudaSuccess ||
        per < 1) {
        cudaGetLastError();
        return;
    }
    ctx->xtma_grid = nsm * per;
    ctx->xtma_state = 1;
}

// x-forward over `rows` rows
template <typename T>
int run_xfwd(mm_ctx* ctx, const T* in, long in_ld, int nin, const T* Ms, T ms, long ms_rows, C_t<T>* out,
             long rows, const C_t<T>* twL, const C_t<T>* twP, int Px) {
    if (!pow2(Px) && Px > kBlueMin && ctx->blue_x.P == Px) {
        KernelTimer kt(ctx, MM_K_XFWD);
        const BlueArrays<T> ba = blue_arrays<T>(ctx->blue_x);
        const int M = ctx->blue_x.M, B = blue_lines(M, sizeof(C_t<T>));
        const size_t smem = (size_t)B * M * sizeof(C_t<T>);
        int rc = set_smem(ctx, (const void*)k_xfwd_blue<T>, smem);
        if (rc) return rc;
        k_xfwd_blue<T><<<(unsigned)((rows + B - 1) / B), block_threads(B * M / 8), smem, ctx->stream>>>(
            in, in_ld, nin, Ms, ms, ms_rows, out, ctx->Hs, ctx->Hx, rows, ilog2(M), ilog2(B), ba.chirp, ba.filt, ba.tw);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    if (!pow2(Px)) {
        KernelTimer kt(ctx, MM_K_XFWD);
        const long n = rows * ctx->Hx;
        k_xfwd_direct<T><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(in, in_ld, nin, Ms, ms, ms_rows, out,
                                                                               ctx->Hs, ctx->Hx, Px, rows, twP);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    KernelTimer kt(ctx, MM_K_XFWD);
    if (Px == 1) {
        k_x1fwd<T><<<(unsigned)((rows + 255) / 256), 256, 0, ctx->stream>>>(in, Ms, ms, ms_rows, out, ctx->Hs, rows);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    const int L = Px / 2;
    if constexpr (sizeof(T) == 4) {
        if (in_ld == L && nin == L && L >= 64) {
            bool done = false;
            int rc = try_xfwd_reg(ctx, in, Ms, ms, ms_rows, out, rows, twL, twP, L, &done);
            if (done) return rc;
        }
    }
    const int B = x_rows_per_block(L);
    size_t smem = (size_t)L * B * sizeof(C_t<T>);
    auto fn = nin <= L ? k_xfwd<T, T, true> : k_xfwd<T, T, false>;
    int rc = set_smem(ctx, (const void*)fn, smem);
    if (rc) return rc;
    fn<<<(unsigned)((rows + B - 1) / B), block_threads(B * L / 8), smem, ctx->stream>>>(
        in, in_ld, nin, Ms, ms, ms_rows, out, ctx->Hs, ilog2(L), rows, ilog2(B), twL, twP);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

// FP32 four-step column transform when L = L1 x L2 is one of the tuned sizes
// and the pruning is the product path's (nin = L/2 forward, nout = L/2 inverse)
template <int L1, int L2, int DIR>
int launch_cols_reg(mm_ctx* ctx, const float2* in, float2* out, int nplanes, ColGeom g, const float2* tw, int c0,
                    int c1) {
    constexpr int L = L1 * L2;
    constexpr int B = 8;   // 64-byte row segments: 15 % faster than 4 columns at L = 1024
    const size_t smem = (size_t)L * B * sizeof(float2);
    auto fn = k_cols_reg<L1, L2, DIR, (DIR < 0), (DIR > 0)>;
    int rc = set_smem(ctx, (const void*)fn, smem);
    if (rc) return rc;
    dim3 grid((unsigned)((c1 - c0 + B - 1) / B), (unsigned)nplanes);
    fn<<<grid, B * (L1 > L2 ? L1 : L2), smem, ctx->stream>>>(in, out, c0, c1, 3, g, tw);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <int DIR>
int try_cols_reg(mm_ctx* ctx, const float2* in, float2* out, int L, int nplanes, ColGeom g, const float2* tw,
                 bool* done, int c0, int c1) {
    *done = true;
    switch (L) {
        case 64: return launch_cols_reg<8, 8, DIR>(ctx, in, out, nplanes, g, tw, c0, c1);
        case 128: return launch_cols_reg<16, 8, DIR>(ctx, in, out, nplanes, g, tw, c0, c1);
        case 256: return launch_cols_reg<16, 16, DIR>(ctx, in, out, nplanes, g, tw, c0, c1);
        case 512: return launch_cols_reg<32, 16, DIR>(ctx, in, out, nplanes, g, tw, c0, c1);
        case 1024: return launch_cols_reg<32, 32, DIR>(ctx, in, out, nplanes, g, tw, c0, c1);
        default: *done = false; return MM_OK;
    }
}

// TMA-fed y passes: descriptors of the pass inputs bufA ([3 nz][ny][Hs]
// complex, the x pass's output) and bufB ([3 nz][Py][Hs], the z pass's
// output), encoded once per context, and the persistent grid of each
// direction (SMs x resident blocks).  Any failure leaves the register passes.
template <int L1, int L2, int DIR>
constexpr auto cols_tma_fn() {
    return k_cols_tma<L1, L2, DIR, (DIR < 0), (DIR > 0)>;
}
template <int L1, int L2>
size_t cols_tma_smem() {
    return (size_t)kYStages * L1 * L2 * kYB * sizeof(float2) + kYStages * sizeof(uint64_t) + 128;
}

template <int L1, int L2>
int ymaps_prepare_t(mm_ctx* ctx) {
    ctx->ymap_state = -1;
    const size_t smem = cols_tma_smem<L1, L2>();
    const void* fns[2] = {(const void*)cols_tma_fn<L1, L2, -1>(), (const void*)cols_tma_fn<L1, L2, +1>()};
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return MM_OK;
    }
    for (int d = 0; d < 2; ++d) {
        int per_sm = 0;
        if (cudaFuncSetAttribute(fns[d], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[d], kYB * (L1 > L2 ? L1 : L2), smem) !=
                cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            return MM_OK;
        }
        ctx->ymap_grid[d] = nsm * per_sm;
    }
    const uint64_t Hs = (uint64_t)ctx->Hs, planes = 3ull * ctx->nz;
    const uint64_t rows[2] = {(uint64_t)ctx->ny, (uint64_t)ctx->Py};
    void* bases[2] = {ctx->bufA, ctx->bufB};
    for (int d = 0; d < 2; ++d) {
        const uint32_t box_rows = (uint32_t)(rows[d] < 256 ? rows[d] : 256);
        if (!tma_encode_3d(ctx->ymap[d], bases[d], 2 * Hs, rows[d], planes, Hs * sizeof(float2),
                           rows[d] * Hs * sizeof(float2), 2 * kYB, box_rows, 1))
            return MM_OK;
    }
    ctx->ymap_state = 1;
    return MM_OK;
}

// the TMA-fed pass when the context qualifies (FP32, plain mode, Py = 512 or
// 1024, the context's own buffers in the product geometry); *done = false
// leaves the register passes
template <int DIR>
int try_cols_tma(mm_ctx* ctx, const float2* in, float2* out, int L, int nplanes, const ColGeom& g, const float2* tw,
                 bool* done) {
    *done = false;
    if (ctx->fft_mode != 0 || (L != 512 && L != 1024) || ctx->Py != L) return MM_OK;
    const bool canonical = DIR < 0 ? ((const void*)in == ctx->bufA && (void*)out == ctx->bufB &&
                                      g.in_inner == (long)ctx->ny * ctx->Hs && g.out_inner == (long)L * ctx->Hs)
                                   : ((const void*)in == ctx->bufB && (void*)out == ctx->bufA &&
                                      g.in_inner == (long)L * ctx->Hs && g.out_inner == (long)ctx->ny * ctx->Hs);
    if (!canonical || nplanes != 3 * ctx->nz || g.n_inner != nplanes || g.in_outer != 0 || g.out_outer != 0 ||
        g.rs_in != ctx->Hs || g.rs_out != ctx->Hs)
        return MM_OK;
    if (ctx->ymap_state == 0) {
        int rc = L == 1024 ? ymaps_prepare_t<32, 32>(ctx) : ymaps_prepare_t<32, 16>(ctx);
        if (rc) return rc;
    }
    if (ctx->ymap_state != 1) return MM_OK;
    alignas(64) CUtensorMap map;
    std::memcpy(&map, ctx->ymap[DIR < 0 ? 0 : 1], sizeof(map));
    const int ntx = (ctx->Hx + kYB - 1) / kYB, ntiles = ntx * nplanes;
    const int grid = ctx->ymap_grid[DIR < 0 ? 0 : 1] < ntiles ? ctx->ymap_grid[DIR < 0 ? 0 : 1] : ntiles;
    int* status = &ctx->ctl->status;
    if (L == 1024) {
        auto fn = cols_tma_fn<32, 32, DIR>();
        fn<<<grid, kYB * 32, cols_tma_smem<32, 32>(), ctx->stream>>>(map, out, ctx->Hx, ntx, ntiles, g.rs_out,
                                                                     g.out_inner, tw, status);
    } else {
        auto fn = cols_tma_fn<32, 16, DIR>();
        fn<<<grid, kYB * 32, cols_tma_smem<32, 16>(), ctx->stream>>>(map, out, ctx->Hx, ntx, ntiles, g.rs_out,
                                                                     g.out_inner, tw, status);
    }
    *done = true;
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <typename T, int DIR>
int run_cols(mm_ctx* ctx, const C_t<T>* in, C_t<T>* out, int L, int nin, int nout, int nplanes, ColGeom g,
             const C_t<T>* tw) {
    KernelTimer kt(ctx, DIR < 0 ? MM_K_YFWD : MM_K_YINV);
    if (!pow2(L) && L > kBlueMin && ctx->blue_y.P == L) {
        if ((const void*)in == (const void*)out) return fail(ctx, MM_ERR_INVALID_ARG, "Bluestein pass needs out != in");
        const BlueArrays<T> ba = blue_arrays<T>(ctx->blue_y);
        const int M = ctx->blue_y.M, B = blue_lines(M, sizeof(C_t<T>));
        const size_t smem = (size_t)B * M * sizeof(C_t<T>);
        int rc = set_smem(ctx, (const void*)k_cols_blue<T, DIR>, smem);
        if (rc) return rc;
        dim3 grid((unsigned)((ctx->Hx + B - 1) / B), (unsigned)nplanes);
        k_cols_blue<T, DIR><<<grid, block_threads(B * M / 8), smem, ctx->stream>>>(
            in, out, nin, nout, ctx->Hx, ilog2(M), ilog2(B), g, ba.chirp, ba.filt, ba.tw);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    if (!pow2(L)) {
        if ((const void*)in == (const void*)out) return fail(ctx, MM_ERR_INVALID_ARG, "direct DFT pass needs out != in");
        dim3 grid((unsigned)(((long)nout * ctx->Hx + 255) / 256), (unsigned)nplanes);
        k_cols_direct<T, DIR><<<grid, 256, 0, ctx->stream>>>(in, out, L, nin, nout, ctx->Hx, g, tw);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    if constexpr (sizeof(T) == 4) {
        const bool product_pruning = DIR < 0 ? (nin == L / 2 && nout == L) : (nin == L && nout == L / 2);
        if (product_pruning && ctx->fft_mode != 0 && (L == 512 || L == 1024))
            return tc_cols(ctx, in, out, L, DIR, nplanes, g, tw);
        if (product_pruning) {
            bool done = false;
            int rc = try_cols_tma<DIR>(ctx, in, out, L, nplanes, g, tw, &done);
            if (done || rc) return rc;
            rc = try_cols_reg<DIR>(ctx, in, out, L, nplanes, g, tw, &done, 0, ctx->Hx);
            if (done) return rc;
        }
    }
    const int B = col_tile(L, sizeof(C_t<T>));
    size_t smem = (size_t)L * B * sizeof(C_t<T>);
    const bool hin = 2 * nin <= L, hout = 2 * nout <= L;
    auto fn = hin ? (hout ? k_cols<T, DIR, true, true> : k_cols<T, DIR, true, false>)
                  : (hout ? k_cols<T, DIR, false, true> : k_cols<T, DIR, false, false>);
    int rc = set_smem(ctx, (const void*)fn, smem);
    if (rc) return rc;
    dim3 grid((unsigned)((ctx->Hx + B - 1) / B), (unsigned)nplanes);
    fn<<<grid, block_threads(B * L / 8), smem, ctx->stream>>>(in, out, ilog2(L), nin, nout, ctx->Hx,
                                                                          ilog2(B), g, tw);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <int PZ>
int launch_zconv_reg_t(mm_ctx* ctx, float2* buf, const float* kern, int c0, int c1) {
    constexpr int PZ2 = PZ / 2 + 1;
    const size_t smem = (size_t)3 * PZ * kZB * sizeof(float2) + (size_t)6 * PZ2 * kZB * sizeof(float);
    if (c0 % 4) return fail(ctx, MM_ERR_INVALID_ARG, "z pass: first column %d not a multiple of 4", c0);
    int rc = set_smem(ctx, (const void*)k_zconv_reg<PZ>, smem);
    if (rc) return rc;
    dim3 grid((unsigned)((c1 - c0 + kZB - 1) / kZB), (unsigned)ctx->Py);
    k_zconv_reg<PZ><<<grid, 3 * kZB, smem, ctx->stream>>>(buf, kern, ctx->Py, ctx->Hs, c0, c1, ctx->Py2);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int launch_zconv_reg(mm_ctx* ctx, float2* buf, const float* kern, int c0, int c1) {
    switch (ctx->Pz) {
        case 1: return launch_zconv_reg_t<1>(ctx, buf, kern, c0, c1);
        case 2: return launch_zconv_reg_t<2>(ctx, buf, kern, c0, c1);
        case 4: return launch_zconv_reg_t<4>(ctx, buf, kern, c0, c1);
        case 8: return launch_zconv_reg_t<8>(ctx, buf, kern, c0, c1);
        case 16: return launch_zconv_reg_t<16>(ctx, buf, kern, c0, c1);
        default: return launch_zconv_reg_t<32>(ctx, buf, kern, c0, c1);
    }
}


// unit = true: the same convolution with Ms = 1 everywhere (H = -N * m),
// the transpose needed by the adjoint
template <typename T>
int xinv_pass(mm_ctx* ctx, const C_t<T>* xin, T* H, long rows);

template <typename T>
int apply(mm_ctx* ctx, const T* m, T* H, bool unit = false) {
    using C = C_t<T>;
    const long plane = (long)ctx->ny * ctx->nx;
    const long rows = 3L * ctx->nz * ctx->ny;
    C* A = (C*)ctx->bufA;
    C* Bf = (C*)ctx->bufB;
    C* xout = ctx->Py == 1 ? Bf : A;
    const T* Ms = (ctx->has_Ms_cell && !unit) ? (const T*)ctx->Ms_cell : nullptr;
    int rc;
    // K2
    rc = run_xfwd<T>(ctx, m, ctx->nx, ctx->nx, Ms, unit ? (T)1 : (T)ctx->Ms, (long)ctx->nz * ctx->ny, xout, rows,
                     table<T>(ctx, ctx->tw.off_lx), table<T>(ctx, ctx->tw.off_px), ctx->Px);
    if (rc) return rc;
    (void)plane;
    if (sizeof(T) == 4 && ctx->fft_mode == MM_FFT_F4) {
        // K3-K5 fused over kx planes, in place on the x pass's spectrum
        if ((rc = f4_yzy(ctx, A))) return rc;
        return xinv_pass<T>(ctx, A, H, rows);
    }
    // K3
    if (ctx->Py > 1) {
        ColGeom g{ctx->Hs, ctx->Hs, 3 * ctx->nz, (long)ctx->ny * ctx->Hs, 0, (long)ctx->Py * ctx->Hs, 0};
        rc = run_cols<T, -1>(ctx, A, Bf, ctx->Py, ctx->ny, ctx->Py, 3 * ctx->nz, g, table<T>(ctx, ctx->tw.off_py));
        if (rc) return rc;
    }
    // K4
    if (sizeof(T) == 4 && ctx->Pz <= 32) {
        KernelTimer kt(ctx, MM_K_ZCONV);
        rc = launch_zconv_reg(ctx, (float2*)Bf, (const float*)ctx->kern, 0, ctx->Hx);
        if (rc) return rc;
    } else {
        KernelTimer kt(ctx, MM_K_ZCONV);
        const int Pz = ctx->Pz;
        const int B = z_tile(Pz, sizeof(C));
        size_t smem = (size_t)3 * Pz * B * sizeof(C) + (size_t)6 * ctx->Pz2 * B * sizeof(T);
        rc = set_smem(ctx, (const void*)k_zconv<T>, smem);
        if (rc) return rc;
        dim3 grid((unsigned)((ctx->Hx + B - 1) / B), (unsigned)(ctx->Py / 2 + 1));
        k_zconv<T><<<grid, block_threads(3 * B * Pz / 8), smem, ctx->stream>>>(
            Bf, (const T*)ctx->kern, ctx->nz, ilog2(Pz), ctx->Py, ctx->Hs, ctx->Hx, ctx->Py2, ctx->Pz2, ilog2(B),
            table<T>(ctx, ctx->tw.off_pz));
        MM_LAUNCH_CHECK(ctx);
    }
    // K5
    if (ctx->Py > 1) {
        ColGeom g{ctx->Hs, ctx->Hs, 3 * ctx->nz, (long)ctx->Py * ctx->Hs, 0, (long)ctx->ny * ctx->Hs, 0};
        rc = run_cols<T, +1>(ctx, Bf, A, ctx->Py, ctx->Py, ctx->ny, 3 * ctx->nz, g, table<T>(ctx, ctx->tw.off_py));
        if (rc) return rc;
    }
    // K6
    return xinv_pass<T>(ctx, ctx->Py == 1 ? Bf : A, H, rows);
}

// K6 from the spectrum xin [3][nz][ny][Hs] to H
template <typename T>
int xinv_pass(mm_ctx* ctx, const C_t<T>* xin, T* H, long rows) {
    using C = C_t<T>;
    int rc;
    const T scale = (T)(1.0 / ((double)ctx->Lx * ctx->Py * ctx->Pz));
    KernelTimer kt(ctx, MM_K_XINV);
    if (!pow2(ctx->Px) && ctx->Px > kBlueMin && ctx->blue_x.P == ctx->Px) {
        const BlueArrays<T> ba = blue_arrays<T>(ctx->blue_x);
        const int M = ctx->blue_x.M, B = blue_lines(M, sizeof(C));
        const size_t smem = (size_t)B * M * sizeof(C);
        rc = set_smem(ctx, (const void*)k_xinv_blue<T>, smem);
        if (rc) return rc;
        k_xinv_blue<T><<<(unsigned)((rows + B - 1) / B), block_threads(B * M / 8), smem, ctx->stream>>>(
            xin, ctx->Hs, H, ctx->nx, rows, scale, ilog2(M), ilog2(B), ba.chirp, ba.filt, ba.tw);
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    if (!pow2(ctx->Px)) {
        const long n = rows * ctx->nx;
        k_xinv_direct<T><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            xin, ctx->Hs, H, ctx->nx, ctx->Px, rows, scale, table<T>(ctx, ctx->tw.off_px));
        MM_LAUNCH_CHECK(ctx);
        return MM_OK;
    }
    if (ctx->Px == 1) {
        k_x1inv<T><<<(unsigned)((rows + 255) / 256), 256, 0, ctx->stream>>>(xin, ctx->Hs, H, rows, scale);
        MM_LAUNCH_CHECK(ctx);
    } else {
        const int L = ctx->Lx;
        if constexpr (sizeof(T) == 4) {
            if (L == 512 && ctx->Hs == kXHs) {
                if (ctx->xtma_state == 0) xtma_prepare(ctx);
                if (ctx->xtma_state == 1) {
                    const int ntiles = (int)((rows + kXB - 1) / kXB);
                    const int grid = ctx->xtma_grid < ntiles ? ctx->xtma_grid : ntiles;
                    k_xinv_tma<<<grid, 128, kXinvTmaSmem, ctx->stream>>>(
                        (const float2*)xin, (float*)H, rows, ntiles, (float)scale,
                        (const float2*)table<T>(ctx, ctx->tw.off_lx), (const float2*)table<T>(ctx, ctx->tw.off_px),
                        &ctx->ctl->status);
                    MM_LAUNCH_CHECK(ctx);
                    return MM_OK;
                }
            }
            bool done = false;
            if (L >= 64) {
                rc = try_xinv_reg(ctx, (const float2*)xin, (float*)H, rows, (float)scale,
                                  (const float2*)table<T>(ctx, ctx->tw.off_lx), (const float2*)table<T>(ctx, ctx->tw.off_px),
                                  L, &done);
                if (done) return rc;
            }
        }
        const int B = x_rows_per_block(L);
        size_t smem = (size_t)L * B * sizeof(C);
        rc = set_smem(ctx, (const void*)k_xinv<T>, smem);
        if (rc) return rc;
        k_xinv<T><<<(unsigned)((rows + B - 1) / B), block_threads(B * L / 8), smem, ctx->stream>>>(
            xin, ctx->Hs, H, ctx->nx, ilog2(L), rows, ilog2(B), scale, table<T>(ctx, ctx->tw.off_lx),
            table<T>(ctx, ctx->tw.off_px));
        MM_LAUNCH_CHECK(ctx);
    }
    return MM_OK;
}

template <typename T>
int setup(mm_ctx* ctx) {
    const long gsize = (long)ctx->Px * ctx->Py * ctx->Pz;
    const long csize = (long)ctx->Pz * ctx->Py * ctx->Hs;
    const long fsize = (long)(ctx->nx + 1) * (ctx->ny + 1) * (ctx->nz + 1);
    double* grid = nullptr;
    double2* X = nullptr;
    double2* fg = nullptr;
    double* oct = nullptr;
    double2* X2 = nullptr;   // out-of-place target of a direct (non-power-of-two) y transform
    int rc = MM_OK;
    auto cleanup = [&]() {
        cudaFree(grid);
        cudaFree(X);
        cudaFree(fg);
        cudaFree(oct);
        cudaFree(X2);
    };
    if (cudaMalloc(&grid, sizeof(double) * gsize) != cudaSuccess || cudaMalloc(&X, sizeof(double2) * csize) != cudaSuccess ||
        cudaMalloc(&fg, sizeof(double2) * fsize) != cudaSuccess || cudaMalloc(&oct, sizeof(double) * 6 * ctx->N) != cudaSuccess ||
        (!pow2(ctx->Py) && cudaMalloc(&X2, sizeof(double2) * csize) != cudaSuccess)) {
        cleanup();
        cudaGetLastError();
        return fail(ctx, MM_ERR_NOMEM, "device allocation for the Newell setup failed");
    }
    const double2* twL = table<double>(ctx, ctx->tw.off_lx);
    const double2* twP = table<double>(ctx, ctx->tw.off_px);
    const long kcomp = (long)ctx->Pz2 * ctx->Py2 * ctx->Hs;
    for (int c = 0; c < 6 && rc == MM_OK; ++c) {
        rc = newell_component(ctx, c, grid, oct + c * ctx->N, fg);
        if (rc) break;
        rc = run_xfwd<double>(ctx, grid, ctx->Px, ctx->Px, nullptr, 1.0, 1, X, (long)ctx->Pz * ctx->Py, twL, twP, ctx->Px);
        if (rc) break;
        double2* Y = X;   // the spectrum after the y transform
        if (ctx->Py > 1) {
            ColGeom g{ctx->Hs, ctx->Hs, ctx->Pz, (long)ctx->Py * ctx->Hs, 0, (long)ctx->Py * ctx->Hs, 0};
            if (X2) Y = X2;
            rc = run_cols<double, -1>(ctx, X, Y, ctx->Py, ctx->Py, ctx->Py, ctx->Pz, g, table<double>(ctx, ctx->tw.off_py));
            if (rc) break;
        }
        if (ctx->Pz > 1) {
            long rs = (long)ctx->Py * ctx->Hs;
            ColGeom g{rs, rs, ctx->Py, ctx->Hs, 0, ctx->Hs, 0};
            rc = run_cols<double, -1>(ctx, Y, Y, ctx->Pz, ctx->Pz, ctx->Pz, ctx->Py, g, table<double>(ctx, ctx->tw.off_pz));
            if (rc) break;
        }
        long total = kcomp;
        k_extract<T><<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(Y, ctx->Py, ctx->Hs, ctx->Hx, ctx->Py2,
                                                                               ctx->Pz2, (T*)ctx->kern + c * kcomp);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) {
            rc = fail(ctx, MM_ERR_CUDA, "k_extract launch failed");
            break;
        }
    }
    if (rc == MM_OK) {
        cudaError_t e = cudaMemcpyAsync(ctx->newell_host, oct, sizeof(double) * 6 * ctx->N, cudaMemcpyDeviceToHost,
                                        ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = fail(ctx, MM_ERR_CUDA, "Newell setup failed: %s", cudaGetErrorString(e));
    } else {
        cudaStreamSynchronize(ctx->stream);
    }
    cleanup();
    return rc;
}

// FP64 context, float-float arithmetic (MM_FFT_FF): the generic passes
// with ff in place of double.  m, Ms and H stay double; the spectra in bufA
// and bufB hold ffc (16 bytes, like double2); the octant and twiddles come
// from their float-float copies (ctx->kern_ff, ctx->tw.ff).  Power-of-two
// Px, Py, Pz only (checked when the mode is set).
int apply_ff(mm_ctx* ctx, const double* m, double* H, bool unit) {
    using C = ffc;
    const long rows = 3L * ctx->nz * ctx->ny;
    C* A = (C*)ctx->bufA;
    C* Bf = (C*)ctx->bufB;
    C* xout = ctx->Py == 1 ? Bf : A;
    const double* Ms = (ctx->has_Ms_cell && !unit) ? (const double*)ctx->Ms_cell : nullptr;
    const ff ms = unit ? ff(1) : ff(ctx->Ms);
    const long ms_rows = (long)ctx->nz * ctx->ny;
    const C* tw = (const C*)ctx->tw.ff;
    int rc;
    {   // K2
        KernelTimer kt(ctx, MM_K_XFWD);
        if (ctx->Px == 1) {
            k_x1fwd<ff, double><<<(unsigned)((rows + 255) / 256), 256, 0, ctx->stream>>>(m, Ms, ms, ms_rows, xout,
                                                                                      ctx->Hs, rows);
        } else {
            const int L = ctx->Px / 2;
            const int B = x_rows_per_block(L);
            const size_t smem = (size_t)L * B * sizeof(C);
            // nin = nx = L: the upper half of each packed line is zero padding
            if ((rc = set_smem(ctx, (const void*)k_xfwd<ff, double, true>, smem))) return rc;
            k_xfwd<ff, double, true><<<(unsigned)((rows + B - 1) / B), block_threads(B * L / 8), smem, ctx->stream>>>(
                m, ctx->nx, ctx->nx, Ms, ms, ms_rows, xout, ctx->Hs, ilog2(L), rows, ilog2(B), tw + ctx->tw.off_lx,
                tw + ctx->tw.off_px);
        }
        MM_LAUNCH_CHECK(ctx);
    }
    // K3
    if (ctx->Py > 1) {
        ColGeom g{ctx->Hs, ctx->Hs, 3 * ctx->nz, (long)ctx->ny * ctx->Hs, 0, (long)ctx->Py * ctx->Hs, 0};
        if ((rc = run_cols<ff, -1>(ctx, A, Bf, ctx->Py, ctx->ny, ctx->Py, 3 * ctx->nz, g, tw + ctx->tw.off_py)))
            return rc;
    }
    {   // K4
        KernelTimer kt(ctx, MM_K_ZCONV);
        const int Pz = ctx->Pz;
        const int B = z_tile(Pz, sizeof(C));
        const size_t smem = (size_t)3 * Pz * B * sizeof(C) + (size_t)6 * ctx->Pz2 * B * sizeof(ff);
        if ((rc = set_smem(ctx, (const void*)k_zconv<ff>, smem))) return rc;
        dim3 grid((unsigned)((ctx->Hx + B - 1) / B), (unsigned)(ctx->Py / 2 + 1));
        k_zconv<ff><<<grid, block_threads(3 * B * Pz / 8), smem, ctx->stream>>>(
            Bf, (const ff*)ctx->kern_ff, ctx->nz, ilog2(Pz), ctx->Py, ctx->Hs, ctx->Hx, ctx->Py2, ctx->Pz2, ilog2(B),
            tw + ctx->tw.off_pz);
        MM_LAUNCH_CHECK(ctx);
    }
    // K5
    if (ctx->Py > 1) {
        ColGeom g{ctx->Hs, ctx->Hs, 3 * ctx->nz, (long)ctx->Py * ctx->Hs, 0, (long)ctx->ny * ctx->Hs, 0};
        if ((rc = run_cols<ff, +1>(ctx, Bf, A, ctx->Py, ctx->Py, ctx->ny, 3 * ctx->nz, g, tw + ctx->tw.off_py)))
            return rc;
    }
    {   // K6
        const C* xin = ctx->Py == 1 ? Bf : A;
        const ff scale = ff(1.0 / ((double)ctx->Lx * ctx->Py * ctx->Pz));
        KernelTimer kt(ctx, MM_K_XINV);
        if (ctx->Px == 1) {
            k_x1inv<ff, double><<<(unsigned)((rows + 255) / 256), 256, 0, ctx->stream>>>(xin, ctx->Hs, H, rows, scale);
        } else {
            const int L = ctx->Lx;
            const int B = x_rows_per_block(L);
            const size_t smem = (size_t)L * B * sizeof(C);
            if ((rc = set_smem(ctx, (const void*)k_xinv<ff, double>, smem))) return rc;
            k_xinv<ff, double><<<(unsigned)((rows + B - 1) / B), block_threads(B * L / 8), smem, ctx->stream>>>(
                xin, ctx->Hs, H, ctx->nx, ilog2(L), rows, ilog2(B), scale, tw + ctx->tw.off_lx, tw + ctx->tw.off_px);
        }
        MM_LAUNCH_CHECK(ctx);
    }
    return MM_OK;
}

// The tensor product of K4 on an unpruned real-to-complex spectrum of the
// whole padded grid, [3][Pz][Py][Hx] complex (x fastest, Hx = Px/2 + 1, the
// layout of a library R2C transform over the three padded axes): one thread
// per k point forms H = -N M from the stored octant with the components'
// parities (xy odd in ky, xz odd in kz, yz odd in both).  In place.
template <typename T>
__global__ void k_kspace_product(C_t<T>* __restrict__ spec, const T* __restrict__ kern, int Pz, int Py, int Hx,
                                 int Hs, int Py2, int Pz2) {
    using C = C_t<T>;
    const long plane = (long)Pz * Py * Hx;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const int kx = (int)(i % Hx);
    const long r = i / Hx;
    const int ky = (int)(r % Py), kz = (int)(r / Py);
    const bool yodd = 2 * ky > Py, zodd = 2 * kz > Pz;
    const int kyp = yodd ? Py - ky : ky, kzp = zodd ? Pz - kz : kz;
    const long kc = (long)Pz2 * Py2 * Hs;
    const long o = ((long)kzp * Py2 + kyp) * Hs + kx;
    const T xx = kern[o], yy = kern[kc + o], zz = kern[2 * kc + o];
    T xy = kern[3 * kc + o], xz = kern[4 * kc + o], yz = kern[5 * kc + o];
    if (yodd) {
        xy = -xy;
        yz = -yz;
    }
    if (zodd) {
        xz = -xz;
        yz = -yz;
    }
    const C mx = spec[i], my = spec[plane + i], mz = spec[2 * plane + i];
    spec[i] = cmk<C>(-(xx * mx.x + xy * my.x + xz * mz.x), -(xx * mx.y + xy * my.y + xz * mz.y));
    spec[plane + i] = cmk<C>(-(xy * mx.x + yy * my.x + yz * mz.x), -(xy * mx.y + yy * my.y + yz * mz.y));
    spec[2 * plane + i] = cmk<C>(-(xz * mx.x + yz * my.x + zz * mz.x), -(xz * mx.y + yz * my.y + zz * mz.y));
}

// float-float copy of an array of doubles (rounding split, once per mode switch)
__global__ void k_split_ff(const double* __restrict__ in, ff* __restrict__ out, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = in[i];
    const float h = __double2float_rn(d);
    out[i] = ff(h, __double2float_rn(d - (double)h));
}

}  // namespace

// Prepares MM_FFT_FF on an FP64 context: float-float copies of the octant
// and of the twiddle tables (kept until the context is destroyed).
int demag_prepare_ff(mm_ctx* ctx) {
    if (ctx->kern_ff && ctx->tw.ff) return MM_OK;
    const long nk = 6L * ctx->Pz2 * ctx->Py2 * ctx->Hs;
    const long nt = 2L * (ctx->tw.off_pz + ctx->Pz);          // doubles in the twiddle table
    if (!ctx->kern_ff) MM_CUDA_CHECK(ctx, cudaMalloc(&ctx->kern_ff, nk * sizeof(ff)));
    if (!ctx->tw.ff) MM_CUDA_CHECK(ctx, cudaMalloc(&ctx->tw.ff, nt * sizeof(ff)));
    k_split_ff<<<(unsigned)((nk + 255) / 256), 256, 0, ctx->stream>>>((const double*)ctx->kern, (ff*)ctx->kern_ff, nk);
    MM_LAUNCH_CHECK(ctx);
    k_split_ff<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>((const double*)ctx->tw.f64, (ff*)ctx->tw.ff, nt);
    MM_LAUNCH_CHECK(ctx);
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int demag_kspace_product(mm_ctx* ctx, void* spec) {
    const long n = (long)ctx->Pz * ctx->Py * ctx->Hx;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (ctx->prec == MM_F64)
        k_kspace_product<double><<<blocks, 256, 0, ctx->stream>>>((double2*)spec, (const double*)ctx->kern, ctx->Pz,
                                                                  ctx->Py, ctx->Hx, ctx->Hs, ctx->Py2, ctx->Pz2);
    else
        k_kspace_product<float><<<blocks, 256, 0, ctx->stream>>>((float2*)spec, (const float*)ctx->kern, ctx->Pz,
                                                                 ctx->Py, ctx->Hx, ctx->Hs, ctx->Py2, ctx->Pz2);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

namespace {
// Bluestein data of one axis (host arithmetic in long double, exact phases)
int blue_axis(mm_ctx* ctx, int P, Blue* bl) {
    if (P <= kBlueMin || pow2(P)) return MM_OK;
    int M = 1;
    while (M < 2 * P - 1) M *= 2;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<double> chirp(2 * (size_t)P), filt(4 * (size_t)M, 0.0), tw(2 * (size_t)M);
    std::vector<long double> cw(M), sw(M);
    for (int m = 0; m < M; ++m) {
        cw[m] = cosl(2.0L * pi * m / M);
        sw[m] = sinl(2.0L * pi * m / M);
        tw[2 * m] = (double)cw[m];
        tw[2 * m + 1] = (double)-sw[m];
    }
    // exp(-i pi n^2 / P) from the exact residue of n^2 mod 2P
    auto ph = [&](long j, long double* c, long double* sn) {
        const long r = (j * j) % (2L * P);
        *c = cosl(pi * r / P);
        *sn = -sinl(pi * r / P);
    };
    for (int n = 0; n < P; ++n) {
        long double c, sn;
        ph(n, &c, &sn);
        chirp[2 * n] = (double)c;
        chirp[2 * n + 1] = (double)sn;
    }
    for (int d = 0; d < 2; ++d) {           // d = 0: DIR -1, filter b[j] = exp(+i pi j^2 / P); d = 1: its conjugate
        std::vector<long double> vr(M, 0.0L), vi(M, 0.0L);
        for (long j = -(P - 1); j <= P - 1; ++j) {
            long double c, sn;
            ph(j, &c, &sn);                 // exp(-i pi j^2 / P)
            const int idx = (int)((j % M + M) % M);
            vr[idx] = c;
            vi[idx] = d == 0 ? -sn : sn;
        }
        for (int k = 0; k < M; ++k) {       // forward DFT of length M, scaled by 1/M
            long double ar = 0.0L, ai = 0.0L;
            for (int j = 0; j < M; ++j) {
                const int m = (int)(((long)j * k) % M);
                ar += vr[j] * cw[m] + vi[j] * sw[m];
                ai += vi[j] * cw[m] - vr[j] * sw[m];
            }
            filt[2 * ((size_t)d * M + k)] = (double)(ar / M);
            filt[2 * ((size_t)d * M + k) + 1] = (double)(ai / M);
        }
    }
    bl->P = P;
    bl->M = M;
    auto up = [&](void** dst, const std::vector<double>& src) -> int {
        MM_CUDA_CHECK(ctx, cudaMalloc(dst, src.size() * sizeof(double)));
        MM_CUDA_CHECK(ctx, cudaMemcpy(*dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
        return MM_OK;
    };
    auto up32 = [&](void** dst, const std::vector<double>& src) -> int {
        std::vector<float> f(src.begin(), src.end());
        MM_CUDA_CHECK(ctx, cudaMalloc(dst, f.size() * sizeof(float)));
        MM_CUDA_CHECK(ctx, cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
        return MM_OK;
    };
    int rc;
    if ((rc = up(&bl->chirp, chirp)) || (rc = up(&bl->filt, filt)) || (rc = up(&bl->tw, tw))) return rc;
    if (ctx->prec == MM_F32 &&
        ((rc = up32(&bl->chirp32, chirp)) || (rc = up32(&bl->filt32, filt)) || (rc = up32(&bl->tw32, tw))))
        return rc;
    return MM_OK;
}
}  // namespace

int blue_prepare(mm_ctx* ctx) {
    int rc = blue_axis(ctx, ctx->Px, &ctx->blue_x);
    if (rc) return rc;
    return blue_axis(ctx, ctx->Py, &ctx->blue_y);
}

int demag_setup(mm_ctx* ctx) {
    return ctx->prec == MM_F64 ? setup<double>(ctx) : setup<float>(ctx);
}

int demag_apply(mm_ctx* ctx, const void* m, void* H) {
    if (ctx->prec == MM_F64) {
        if (ctx->fft_mode == MM_FFT_FF) return apply_ff(ctx, (const double*)m, (double*)H, false);
        return apply<double>(ctx, (const double*)m, (double*)H);
    }
    return apply<float>(ctx, (const float*)m, (float*)H);
}

int demag_apply_unit(mm_ctx* ctx, const void* g, void* H) {
    if (ctx->prec == MM_F64) {
        if (ctx->fft_mode == MM_FFT_FF) return apply_ff(ctx, (const double*)g, (double*)H, true);
        return apply<double>(ctx, (const double*)g, (double*)H, true);
    }
    return apply<float>(ctx, (const float*)g, (float*)H, true);
}

}  // namespace mm

namespace mm {

// cuTensorMapEncodeTiled, looked up once through the runtime (no libcuda link)
bool tma_encode_3d(void* map128, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1, uint64_t s2,
                   uint32_t b0, uint32_t b1, uint32_t b2) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode enc = []() -> Encode {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return (Encode)fn;
    }();
    if (!enc) return false;
    alignas(64) CUtensorMap map;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {s1, s2};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    std::memcpy(map128, &map, sizeof(map));
    return true;
}

}  // namespace mm
