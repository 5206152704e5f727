// Three-pass thin-film demag (MM_FFT_F4): the y forward transform, the z
// transform with the tensor product, and the y inverse transform fused into
// one pass over a kx plane, held on chip in a cluster of four CTAs, so the
// spectrum makes one round trip through HBM between the two x passes
// instead of three (the paper's FFT paragraph in the Implementation section
// describes the padded transforms this reorganises; Eq. 4 is unchanged).
//
// For one kx, the plane holds the 3 x nz lines of length Py = 1024 (ny = 512
// non-zero inputs).  CTA r of the cluster owns the wavenumbers ky = 4 j + r:
//   X[4 j + r] = DFT_256(y_r)[j],  y_r[m] = w^(m r) (x[m] + (-i)^r x[m + 256]),
// with w = exp(-2 pi i / 1024) and x[n] = 0 for n >= 512, so the forward
// transform and the pointwise z convolution need no data of the other
// CTAs.  Back in space,
//   x[n] = sum_r w^(-n r) Z_r[n mod 256],  Z_r = IDFT_256(X_r),
// so after its inverse each CTA writes the outputs of 12 of the 48 lines,
// reading the four Z_r of those lines from the cluster's shared memory.
//
// Per CTA: 768 threads; the 48 lines of 256 values (96 KB) and the z-product
// exchange (96 KB) in shared memory: one CTA per SM.  The z step is the
// parity-split register form (two threads per z line, kz even and odd).
// The Newell octant is re-laid out once for this mode as
// [kx][r][component][kz'][j] with the ky-parity signs applied, so each CTA
// reads its rows contiguously.  Supported mesh: ny = 512, nz = 16 (the
// 512 x 512 x 16 film and others of that ny and nz), FP32.
#include <cooperative_groups.h>

#include "mm_regfft.cuh"

namespace cg = cooperative_groups;

namespace mm {
namespace {

constexpr int kF4Ranks = 4, kF4Threads = 768, kF4NZ = 16, kF4PZ = 32, kF4Lines = 3 * kF4NZ, kF4Len = 256;
constexpr int kF4Tile = 128;                                  // ky per z-step tile
constexpr size_t kF4Smem = (size_t)kF4Lines * kF4Len * sizeof(float2) + (size_t)6 * 16 * kF4Tile * sizeof(float2);

// swizzled position of (k1, t) in a 16 x 16 transpose
__device__ __forceinline__ int sw16(int k1, int t) { return k1 * 16 + (t ^ (k1 & 15)); }

// the octant re-laid out for the fused pass: out[kx][r][comp][kzp][j] =
// sign N_comp(kx, ky = 4 j + r, kzp), sign = -1 for xy and yz when ky > Py/2
__global__ void k_f4_kernel(const float* __restrict__ kern, float* __restrict__ out, int Hx, int Hs, int Py, int Py2,
                            int Pz2) {
    const long total = (long)Hx * kF4Ranks * 6 * Pz2 * kF4Len;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % kF4Len);
        long rest = idx / kF4Len;
        const int kzp = (int)(rest % Pz2);
        rest /= Pz2;
        const int comp = (int)(rest % 6);
        rest /= 6;
        const int r = (int)(rest % kF4Ranks);
        const int kx = (int)(rest / kF4Ranks);
        const int ky = 4 * j + r;
        const bool yodd = 2 * ky > Py;
        const int kyp = yodd ? Py - ky : ky;
        float v = kern[(((long)comp * Pz2 + kzp) * Py2 + kyp) * Hs + kx];
        if (yodd && (comp == 3 || comp == 5)) v = -v;
        out[idx] = v;
    }
}

// phase 1 for CTA rank R: lines l = c nz + z, thread (t, l) holds y_R[t + 16 m1]
template <int R>
__device__ __forceinline__ void f4_forward(const float2* __restrict__ A, float2* D, int kx, int Hs, int l, int t,
                                           const float2* __restrict__ tw1024, const float2* __restrict__ tw256) {
    float2 v[16];
    const float2* col = A + (long)l * 512 * Hs + kx;
    const float2 wt = tw1024[(t * R) & 1023];             // w^(t R)
    static_for<0, 16>([&](auto M1) {
        constexpr int m1 = decltype(M1)::value;
        const int m = t + 16 * m1;
        float2 a = col[(long)m * Hs];
        const float2 b = col[(long)(m + 256) * Hs];
        // (-i)^R b
        if constexpr (R == 0) a = cadd(a, b);
        else if constexpr (R == 1) a = make_float2(a.x + b.y, a.y - b.x);
        else if constexpr (R == 2) a = csub(a, b);
        else a = make_float2(a.x - b.y, a.y + b.x);
        if constexpr (R > 0) {
            // w^(m R) = w^(t R) w^(16 m1 R), the second a 64th root of unity
            constexpr double c = cos2pi((m1 * R) % 64, 64), s = -sin2pi((m1 * R) % 64, 64);
            a = cmul(cmul(a, wt), make_float2((float)c, (float)s));
        }
        v[m1] = a;
    });
    dif<16, -1, false>(v);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
        float2 y = v[dif_pos<16>(k1)];
        if (k1 > 0) y = cmul(y, tw256[t * k1]);
        D[l * kF4Len + sw16(k1, t)] = y;
    }
}

// the product of one kz parity class for component C (octant rows of this
// CTA: K[comp][kzp][j] with the ky signs applied)
template <int Q, int C>
__device__ __forceinline__ void f4_product(float2 (&v)[16], const float2* S, const float* __restrict__ K, int jj,
                                           int j) {
    constexpr int PZ2 = kF4PZ / 2 + 1;
    constexpr int I0 = C == 0 ? 0 : C == 1 ? 3 : 4;
    constexpr int I1 = C == 0 ? 3 : C == 1 ? 1 : 5;
    constexpr int I2 = C == 0 ? 4 : C == 1 ? 5 : 2;
    static_for<0, 16>([&](auto J) {
        constexpr int k = decltype(J)::value;
        constexpr int kz = 2 * k + Q;
        constexpr int kzp = kz <= kF4PZ / 2 ? kz : kF4PZ - kz;
        constexpr bool odd = kz > kF4PZ / 2;
        float a0 = K[(I0 * PZ2 + kzp) * kF4Len + j];
        float a1 = K[(I1 * PZ2 + kzp) * kF4Len + j];
        float a2 = K[(I2 * PZ2 + kzp) * kF4Len + j];
        if constexpr (odd) {
            if constexpr (C == 2) {
                a0 = -a0;
                a1 = -a1;
            } else {
                a2 = -a2;
            }
        }
        const float2 mx = S[((0 * 2 + Q) * 16 + k) * kF4Tile + jj];
        const float2 my = S[((1 * 2 + Q) * 16 + k) * kF4Tile + jj];
        const float2 mz = S[((2 * 2 + Q) * 16 + k) * kF4Tile + jj];
        v[k] = make_float2(-(a0 * mx.x + a1 * my.x + a2 * mz.x), -(a0 * mx.y + a1 * my.y + a2 * mz.y));
    });
}

template <int R>
__device__ __forceinline__ void f4_gather(cg::cluster_group& cluster, float2* D, float2* __restrict__ A, int kx, int Hs,
                                          const float2* __restrict__ tw1024) {
    // CTA R writes lines 12 R .. 12 R + 11: x[m + 256 s] = sum_r w^(-(m + 256 s) r) Z_r[m]
    const float2* Dr[kF4Ranks];
#pragma unroll
    for (int r = 0; r < kF4Ranks; ++r) Dr[r] = cluster.map_shared_rank(D, r);
    for (int e = threadIdx.x; e < 12 * kF4Len; e += blockDim.x) {
        const int l = 12 * R + e / kF4Len, m = e % kF4Len;
        float2 z[kF4Ranks];
#pragma unroll
        for (int r = 0; r < kF4Ranks; ++r) z[r] = Dr[r][l * kF4Len + m];
        float2 lo = z[0], hi = z[0];
#pragma unroll
        for (int r = 1; r < kF4Ranks; ++r) {
            const float2 w = cconj(tw1024[(m * r) & 1023]);          // w^(-m r)
            const float2 p = cmul(z[r], w);
            lo = cadd(lo, p);
            // w^(-256 s r) = i^(s r) for s = 1
            hi = r == 1 ? make_float2(hi.x - p.y, hi.y + p.x) : r == 2 ? csub(hi, p) : make_float2(hi.x + p.y, hi.y - p.x);
        }
        float2* col = A + (long)l * 512 * Hs + kx;
        col[(long)m * Hs] = lo;
        col[(long)(m + 256) * Hs] = hi;
    }
}

__global__ void __cluster_dims__(kF4Ranks, 1, 1) __launch_bounds__(kF4Threads, 1)
    k_f4_yzy(float2* __restrict__ A, const float* __restrict__ kf4, int Hs, const float2* __restrict__ tw1024,
             const float2* __restrict__ tw256) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* D = reinterpret_cast<float2*>(smem_raw);                          // [48][256]
    float2* S = D + kF4Lines * kF4Len;                                        // [3][2][16][128]
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int kx = blockIdx.x / kF4Ranks;
    const int tid = threadIdx.x;
    // ---- phase 1: y forward (this CTA's ky class), 16 threads per line
    {
        const int l = tid / 16, t = tid % 16;
        if (r == 0) f4_forward<0>(A, D, kx, Hs, l, t, tw1024, tw256);
        else if (r == 1) f4_forward<1>(A, D, kx, Hs, l, t, tw1024, tw256);
        else if (r == 2) f4_forward<2>(A, D, kx, Hs, l, t, tw1024, tw256);
        else f4_forward<3>(A, D, kx, Hs, l, t, tw1024, tw256);
        __syncthreads();
        float2 u[16];
        const int k1 = t;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) u[n2] = D[l * kF4Len + sw16(k1, n2)];
        dif<16, -1, false>(u);
        __syncthreads();
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) D[l * kF4Len + k1 + 16 * k2] = u[dif_pos<16>(k2)];
        __syncthreads();
    }
    // ---- phase 2: z transform, product, z inverse, in two tiles of 128 ky
    {
        const int c = tid / (2 * kF4Tile), q = (tid / kF4Tile) & 1, jj = tid % kF4Tile;
        const float* K = kf4 + ((long)kx * kF4Ranks + r) * 6 * (kF4PZ / 2 + 1) * kF4Len;
        for (int j0 = 0; j0 < kF4Len; j0 += kF4Tile) {
            const int j = j0 + jj;
            float2 v[16];
#pragma unroll
            for (int z = 0; z < 16; ++z) v[z] = D[(c * 16 + z) * kF4Len + j];
            if (q == 1) {
                static_for<1, 16>([&](auto N) {
                    constexpr int n = decltype(N)::value;
                    constexpr double cs = cos2pi(n, kF4PZ), sn = -sin2pi(n, kF4PZ);
                    v[n] = cmul(v[n], make_float2((float)cs, (float)sn));
                });
            }
            dif<16, -1, false>(v);
#pragma unroll
            for (int k = 0; k < 16; ++k) S[((c * 2 + q) * 16 + k) * kF4Tile + jj] = v[dif_pos<16>(k)];
            __syncthreads();
            if (q == 0) {
                if (c == 0) f4_product<0, 0>(v, S, K, jj, j);
                else if (c == 1) f4_product<0, 1>(v, S, K, jj, j);
                else f4_product<0, 2>(v, S, K, jj, j);
            } else {
                if (c == 0) f4_product<1, 0>(v, S, K, jj, j);
                else if (c == 1) f4_product<1, 1>(v, S, K, jj, j);
                else f4_product<1, 2>(v, S, K, jj, j);
            }
            dif<16, +1, false>(v);
            __syncthreads();
            if (q == 1) {
                static_for<0, 16>([&](auto N) {
                    constexpr int n = decltype(N)::value;
                    float2 o = v[dif_pos<16>(n)];
                    if constexpr (n > 0) {
                        constexpr double cs = cos2pi(n, kF4PZ), sn = sin2pi(n, kF4PZ);
                        o = cmul(o, make_float2((float)cs, (float)sn));
                    }
                    S[((c * 2 + 1) * 16 + n) * kF4Tile + jj] = o;
                });
            } else {
#pragma unroll
                for (int n = 0; n < 16; ++n) S[((c * 2) * 16 + n) * kF4Tile + jj] = v[dif_pos<16>(n)];
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int z = q * 8 + i;
                D[(c * 16 + z) * kF4Len + j] =
                    cadd(S[((c * 2) * 16 + z) * kF4Tile + jj], S[((c * 2 + 1) * 16 + z) * kF4Tile + jj]);
            }
            __syncthreads();
        }
    }
    // ---- phase 3: inverse 256-point transforms of this CTA's class (16 x 16)
    {
        const int l = tid / 16, t = tid % 16;
        float2 v[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) v[n1] = D[l * kF4Len + t + 16 * n1];
        dif<16, +1, false>(v);
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            float2 y = v[dif_pos<16>(k1)];
            if (k1 > 0) y = cmul(y, cconj(tw256[t * k1]));
            D[l * kF4Len + sw16(k1, t)] = y;
        }
        __syncthreads();
        float2 u[16];
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) u[n2] = D[l * kF4Len + sw16(t, n2)];
        dif<16, +1, false>(u);
        __syncthreads();
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) D[l * kF4Len + t + 16 * k2] = u[dif_pos<16>(k2)];
    }
    cluster.sync();                        // every Z_r of the plane is in place
    if (r == 0) f4_gather<0>(cluster, D, A, kx, Hs, tw1024);
    else if (r == 1) f4_gather<1>(cluster, D, A, kx, Hs, tw1024);
    else if (r == 2) f4_gather<2>(cluster, D, A, kx, Hs, tw1024);
    else f4_gather<3>(cluster, D, A, kx, Hs, tw1024);
    cluster.sync();                        // no CTA leaves while its Z_r is read
}

}  // namespace

bool f4_supported(const mm_ctx* ctx) { return ctx->prec == MM_F32 && ctx->ny == 512 && ctx->nz == kF4NZ; }

int f4_prepare(mm_ctx* ctx) {
    if (ctx->kern_f4) return MM_OK;
    const long n = (long)ctx->Hx * kF4Ranks * 6 * ctx->Pz2 * kF4Len;
    MM_CUDA_CHECK(ctx, cudaMalloc(&ctx->kern_f4, n * sizeof(float)));
    // twiddles exp(-2 pi i m / 1024) and exp(-2 pi i m / 256) for the pass
    std::vector<float2> tw(1024 + 256);
    for (int m = 0; m < 1024; ++m) {
        const long double a = 2.0L * 3.141592653589793238462643383279502884L * m / 1024.0L;
        tw[m] = make_float2((float)cosl(a), (float)-sinl(a));
    }
    for (int m = 0; m < 256; ++m) tw[1024 + m] = tw[4 * m];
    MM_CUDA_CHECK(ctx, cudaMalloc(&ctx->tw_f4, tw.size() * sizeof(float2)));
    MM_CUDA_CHECK(ctx, cudaMemcpy(ctx->tw_f4, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    k_f4_kernel<<<1024, 256, 0, ctx->stream>>>((const float*)ctx->kern, (float*)ctx->kern_f4, ctx->Hx, ctx->Hs, ctx->Py,
                                               ctx->Py2, ctx->Pz2);
    MM_LAUNCH_CHECK(ctx);
    MM_CUDA_CHECK(ctx, cudaFuncSetAttribute(k_f4_yzy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kF4Smem));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

// y forward, z product, y inverse of the spectrum A [3][nz][ny][Hs] in place
int f4_yzy(mm_ctx* ctx, void* A) {
    KernelTimer kt(ctx, MM_K_ZCONV);
    const float2* tw = (const float2*)ctx->tw_f4;
    k_f4_yzy<<<(unsigned)(kF4Ranks * ctx->Hx), kF4Threads, kF4Smem, ctx->stream>>>(
        (float2*)A, (const float*)ctx->kern_f4, ctx->Hs, tw, tw + 1024);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace mm
