// Fourier neural operator surrogate of the demagnetisation field (2-D films,
// nz = 1) with hand-written forward, backward and Adam kernels.
//
// Network (per sample, grid NY x NX, width W, MX x MY retained modes with
// kx in [0, MX) and ky in [0, MX) U [NY - MX, NY)):
//   v0 = P m + p                                  (lift, 1x1, 3 -> W)
//   a_l = W_l v_l + b_l + IDFT_x IDFT_y (R_l . DFT_y DFT_x v_l),
//   v_{l+1} = GELU(a_l) (l < L-1), v_L = a_{L-1}
//   h = Q v_L + q                                 (projection, 1x1, W -> 3)
// trained on h = H_demag / Ms.  DFT_x keeps kx < MX of the real input;
// IDFT_x is the matching truncated real inverse
// z(x) = sum_kx c_kx Re(u_kx e^{2 pi i kx x / NX}) / (NX NY), c_0 = 1, else 2.
// R_l[co][ci][ky][kx] are complex per-mode channel mixers.  Activations are
// stored as BF16 (or FP32) and every contraction accumulates in FP32.
//
// Backward uses the adjoints under the real inner product: the adjoint of a
// complex-linear map is its conjugate transpose (DFT_y <-> IDFT_y with
// flipped sign, T = R S -> dS = R^H dT, dR = dT S^H), the adjoint of
// DFT_x on real input is Re(sum dA e^{+i theta}), that of IDFT_x is
// c_kx / (NX NY) sum_x g e^{-i theta}.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdlib>
#include <vector>

#include "mm_internal.cuh"
#include "mm_tcgen05.cuh"

struct mm_fno {
    int nx, ny, W, M, L, store_bf16, max_batch, device;
    cudaStream_t stream;
    long P;             // pixels
    int MY, K;          // ky count (2 M), modes per channel (MY * M)
    long nparams;
    float* params;      // master weights, FP32
    float* grads;
    float* adam_m;
    float* adam_v;
    // offsets into params
    long o_P, o_p, o_Q, o_q;
    std::vector<long> o_W, o_b, o_R;
    // activations (storage type) and spectral buffers
    void* v;            // [L+1][B][W][P]  v_0 .. v_L
    void* a;            // [L][B][W][P]    pre-activations
    float2* S;          // [L][B][W][K]    retained spectra of v_l
    float2* A;          // [B][W][NY][M]   x-transform scratch
    float2* T;          // [B][W][K]
    float2* U;          // [B][W][NY][M]
    void* dv;           // [2][B][W][P]    ping-pong cotangents (FP32)
    float2* twx;        // [M][NX]  e^{-2 pi i kx x / NX}
    float2* twy;        // [MY][NY] e^{-2 pi i ky y / NY}
    float* basis;       // [2M][NX] inverse-x basis c_kx (cos, -sin) / (NX NY), c_0 = 1, else 2
    double* red;        // loss reduction scratch [2][B]
    unsigned char* xbimg;   // tensor-core x transform: twiddle operand image [NX/64][hi, lo][NP x 64] BF16
    int xNP;            // its N (2M rounded up to 16)
    float out_scale;    // multiply h by this on output (Ms inside relax)
    std::string err;
};

namespace mm {
namespace {

template <typename S> __device__ __forceinline__ float ld(const S* p, long i);
template <> __device__ __forceinline__ float ld<float>(const float* p, long i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, long i) {
    return __bfloat162float(p[i]);
}
template <typename S> __device__ __forceinline__ void st(S* p, long i, float v);
template <> __device__ __forceinline__ void st<float>(float* p, long i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16* p, long i, float v) {
    p[i] = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// ky index of retained row r: 0..M-1 then NY-M..NY-1
__device__ __forceinline__ int ky_of(int r, int M, int NY) { return r < M ? r : NY - 2 * M + r; }

// 1x1 channel map: Y[b][co][p] = sum_ci Wt[co][ci] X[b][ci][p] + bias[co] (times scale)
template <typename SI, typename SO>
__global__ void k_chan(const SI* __restrict__ X, const float* __restrict__ Wt, const float* __restrict__ bias,
                       SO* __restrict__ Y, int Ci, int Co, long P, int B, float scale, int transpose) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)B * P) return;
    const int b = (int)(idx / P);
    const long p = idx % P;
    float x[32];   // unrolled to the maximum width so that it stays in registers
#pragma unroll
    for (int ci = 0; ci < 32; ++ci) x[ci] = ci < Ci ? ld(X, ((long)b * Ci + ci) * P + p) : 0.f;
    for (int co = 0; co < Co; ++co) {
        float acc = bias ? bias[co] : 0.f;
#pragma unroll
        for (int ci = 0; ci < 32; ++ci)
            if (ci < Ci) acc += (transpose ? Wt[ci * Co + co] : Wt[co * Ci + ci]) * x[ci];
        st(Y, ((long)b * Co + co) * P + p, acc * scale);
    }
}

// A[row][kx] = sum_x X[row][x] e^{-2 pi i kx x / NX} * colscale(kx); rows = B W NY.
// A GEMM of the rows against the twiddle table: 64 rows per block, x in
// chunks of 32 staged in shared memory with the matching twiddles; thread t
// owns row t / 4 and the modes kx = t % 4 + 4 j (M <= 32).
constexpr int kDxRows = 64, kDxChunk = 32, kMaxModes = 32;

template <typename SI>
__global__ void __launch_bounds__(256) k_dft_x(const SI* __restrict__ X, float2* __restrict__ A,
                                               const float2* __restrict__ twx, long rows, int NX, int M, float scale0,
                                               float scale1) {
    __shared__ float xs[kDxRows][kDxChunk + 1];
    __shared__ float2 ts[kDxChunk][kMaxModes];
    const int tid = threadIdx.x;
    const long r0 = (long)blockIdx.x * kDxRows;
    const int rl = tid >> 2, g = tid & 3;
    float2 acc[kMaxModes / 4];
#pragma unroll
    for (int j = 0; j < kMaxModes / 4; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int x0 = 0; x0 < NX; x0 += kDxChunk) {
        for (int e = tid; e < kDxRows * kDxChunk; e += blockDim.x) {
            const int r = e / kDxChunk, x = e % kDxChunk;
            const long row = r0 + r;
            xs[r][x] = (row < rows && x0 + x < NX) ? ld(X, row * NX + x0 + x) : 0.f;
        }
        for (int e = tid; e < M * kDxChunk; e += blockDim.x) {
            const int k = e / kDxChunk, x = e % kDxChunk;
            ts[x][k] = x0 + x < NX ? twx[(long)k * NX + x0 + x] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int x = 0; x < kDxChunk; ++x) {
            const float v = xs[rl][x];
#pragma unroll
            for (int j = 0; j < kMaxModes / 4; ++j) {
                const int k = g + 4 * j;
                if (k < M) {
                    const float2 w = ts[x][k];
                    acc[j].x += v * w.x;
                    acc[j].y += v * w.y;
                }
            }
        }
        __syncthreads();
    }
    const long row = r0 + rl;
    if (row < rows) {
#pragma unroll
        for (int j = 0; j < kMaxModes / 4; ++j) {
            const int k = g + 4 * j;
            if (k < M) {
                const float sc = k == 0 ? scale0 : scale1;
                A[row * M + k] = make_float2(acc[j].x * sc, acc[j].y * sc);
            }
        }
    }
}

// along y between NY rows and the 2M retained rows; fwd: out[r] = sum_y in[y]
// e^{sign 2 pi i ky(r) y / NY} (NY -> 2M); adjoint direction (2M -> NY):
// out[y] = sum_r in[r] e^{sign 2 pi i ky(r) y / NY}
__global__ void k_dft_y(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ twy, int BW,
                        int NY, int M, int to_modes, float sign) {
    const int MY = 2 * M;
    const long nout = (long)BW * (to_modes ? MY : NY) * M;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nout) return;
    const int kx = (int)(idx % M);
    const long rest = idx / M;
    const int nrow_out = to_modes ? MY : NY;
    const int r = (int)(rest % nrow_out);
    const long bw = rest / nrow_out;
    float re = 0.f, im = 0.f;
    const int nin = to_modes ? NY : MY;
    for (int j = 0; j < nin; ++j) {
        const int y = to_modes ? j : r;
        const int mr = to_modes ? r : j;
        float2 w = twy[mr * NY + y];             // e^{-2 pi i ky y / NY}
        w.y *= -sign;                            // sign -1: as tabulated, +1: conjugate
        const float2 v = in[(bw * nin + j) * M + kx];
        re += v.x * w.x - v.y * w.y;
        im += v.x * w.y + v.y * w.x;
    }
    out[idx] = make_float2(re, im);
}

// NY -> 2M retained rows with the sum over y split over 8 lanes (shuffle
// reduction): out[bw][r][kx] = sum_y in[bw][y][kx] e^{sign 2 pi i ky(r) y / NY}
__global__ void k_dft_y_modes(const float2* __restrict__ in, float2* __restrict__ out,
                              const float2* __restrict__ twy, int BW, int NY, int M, float sign) {
    const int MY = 2 * M;
    const long nout = (long)BW * MY * M;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long idx = gid >> 3;
    const int lane = (int)(gid & 7);
    float re = 0.f, im = 0.f;
    if (idx < nout) {
        const int kx = (int)(idx % M);
        const long rest = idx / M;
        const int r = (int)(rest % MY);
        const long bw = rest / MY;
        for (int y = lane; y < NY; y += 8) {
            float2 w = twy[(long)r * NY + y];     // e^{-2 pi i ky y / NY}
            w.y *= -sign;
            const float2 v = in[(bw * NY + y) * M + kx];
            re += v.x * w.x - v.y * w.y;
            im += v.x * w.y + v.y * w.x;
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (idx < nout && lane == 0) out[idx] = make_float2(re, im);
}

// T[b][co][k] = sum_ci R[co][ci][k] S[b][ci][k]; adjoint: S' = sum_co conj(R[co][ci]) T
__global__ void k_mix(const float2* __restrict__ in, const float2* __restrict__ R, float2* __restrict__ out, int B, int W,
                      int K, int adjoint) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)B * W * K) return;
    const int k = (int)(idx % K);
    const int o = (int)((idx / K) % W);
    const int b = (int)(idx / ((long)K * W));
    float re = 0.f, im = 0.f;
    for (int i = 0; i < W; ++i) {
        float2 r = adjoint ? R[((long)i * W + o) * K + k] : R[((long)o * W + i) * K + k];
        if (adjoint) r.y = -r.y;
        const float2 v = in[((long)b * W + i) * K + k];
        re += r.x * v.x - r.y * v.y;
        im += r.x * v.y + r.y * v.x;
    }
    out[idx] = make_float2(re, im);
}

// dR[co][ci][k] += sum_b dT[b][co][k] conj(S[b][ci][k])
__global__ void k_mix_grad(const float2* __restrict__ dT, const float2* __restrict__ S, float2* __restrict__ dR, int B,
                           int W, int K) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)W * W * K) return;
    const int k = (int)(idx % K);
    const int ci = (int)((idx / K) % W);
    const int co = (int)(idx / ((long)K * W));
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
        const float2 g = dT[((long)b * W + co) * K + k];
        const float2 s = S[((long)b * W + ci) * K + k];
        re += g.x * s.x + g.y * s.y;
        im += g.y * s.x - g.x * s.y;
    }
    dR[idx].x += re;
    dR[idx].y += im;
}

// a[b][co][p] = W v + bias + IDFT_x(U)[co][y][x];  v_next = GELU(a) or a.
// Per (y, b) row and tile of 256 x, one GEMM with K = W + 2M:
//   a[co][x] = bias[co] + sum_k Am[co][k] Bm[k][x],
//   Am = [W | Re U, Im U],  Bm = [v rows ; basis rows],
// the basis rows holding c_kx Re / Im of e^{-2 pi i kx x / NX} / (NX NY)
// (Re(u conj(w)) = u.x w.x + u.y w.y).  Both operands in shared memory,
// each thread an 8 (co) x 4 (x) register tile.
constexpr int kLoTile = 256;

template <typename SS>
__global__ void __launch_bounds__(256) k_layer_out(const SS* __restrict__ v, const float2* __restrict__ U,
                                                   const float* __restrict__ Wt, const float* __restrict__ bias,
                                                   const float* __restrict__ basis, SS* __restrict__ a_out,
                                                   SS* __restrict__ v_next, int B, int W, int NY, int NX, int M,
                                                   int last) {
    constexpr int KMAX = 32 + 2 * kMaxModes;
    __shared__ float As[32][KMAX + 1];
    extern __shared__ __align__(16) float Bs[];           // [K][kLoTile]
    const int y = blockIdx.x, b = blockIdx.y, x0 = blockIdx.z * kLoTile;
    const int K = W + 2 * M;
    const long P = (long)NY * NX;
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * K; e += blockDim.x) {
        const int co = e / K, k = e % K;
        float val = 0.f;
        if (co < W) {
            if (k < W) {
                val = Wt[co * W + k];
            } else {
                const int kx = (k - W) >> 1;
                const float2 u = U[(((long)b * W + co) * NY + y) * M + kx];
                val = ((k - W) & 1) ? u.y : u.x;
            }
        }
        As[co][k] = val;
    }
    for (int e = tid; e < K * kLoTile; e += blockDim.x) {
        const int k = e / kLoTile, x = e % kLoTile;
        float val = 0.f;
        if (x0 + x < NX)
            val = k < W ? ld(v, ((long)b * W + k) * P + (long)y * NX + x0 + x) : basis[(long)(k - W) * NX + x0 + x];
        Bs[k * kLoTile + x] = val;
    }
    __syncthreads();
    const int cg = tid >> 6, xg = tid & 63;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k = 0; k < K; ++k) {
        float av[8], bv[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = As[8 * cg + i][k];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[k * kLoTile + xg + 64 * j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int co = 8 * cg + i;
        if (co >= W) continue;
        const float bb = bias[co];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + xg + 64 * j;
            if (x >= NX) continue;
            const float val = acc[i][j] + bb;
            const long o = ((long)b * W + co) * P + (long)y * NX + x;
            st(a_out, o, val);
            st(v_next, o, last ? val : gelu(val));
        }
    }
}

inline size_t layer_out_smem(int W, int M) { return (size_t)(W + 2 * M) * kLoTile * sizeof(float); }

// da = dvn * GELU'(a) (or dvn for the last layer), FP32 in place
template <typename SS>
__global__ void k_gelu_bwd(float* __restrict__ dv, const SS* __restrict__ a, long n, int last) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || last) return;
    dv[i] *= gelu_grad(ld(a, i));
}

// dX[row][x] (+)= Re(sum_kx dA[row][kx] e^{+2 pi i kx x / NX})
__global__ void k_dft_x_adj(const float2* __restrict__ dA, float* __restrict__ dX, const float2* __restrict__ twx,
                            long rows, int NX, int M, int accumulate) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * NX) return;
    const long row = idx / NX;
    const int x = (int)(idx % NX);
    float s = 0.f;
    for (int kx = 0; kx < M; ++kx) {
        const float2 g = dA[row * M + kx];
        const float2 w = twx[kx * NX + x];
        s += g.x * w.x + g.y * w.y;             // Re(g conj(w))
    }
    dX[idx] = accumulate ? dX[idx] + s : s;
}

// dW[co][ci] += sum_{b,p} dY[b][co][p] X[b][ci][p]; db[co] += sum dY (the
// column ci == Ci).  Blocks walk chunks of 128 pixels of one sample, stage
// dY and X for the chunk in shared memory and accumulate their share of the
// Co (Ci + 1) outputs in registers; one atomic add per output per block.
constexpr int kWgChunk = 128;

template <typename SX>
__global__ void __launch_bounds__(256) k_wgrad(const float* __restrict__ dY, const SX* __restrict__ X,
                                               float* __restrict__ dW, float* __restrict__ db, int Co, int Ci, long P,
                                               int B) {
    __shared__ float ys[32][kWgChunk + 1];
    __shared__ float xs[32][kWgChunk + 1];
    constexpr int J = (32 * 33 + 255) / 256;
    const int nout = Co * (Ci + 1);
    float acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = 0.f;
    const long cps = (P + kWgChunk - 1) / kWgChunk;       // chunks per sample
    for (long c = blockIdx.x; c < (long)B * cps; c += gridDim.x) {
        const int b = (int)(c / cps);
        const long p0 = (c % cps) * kWgChunk;
        for (int e = threadIdx.x; e < Co * kWgChunk; e += blockDim.x) {
            const int co = e / kWgChunk, pp = e % kWgChunk;
            ys[co][pp] = p0 + pp < P ? dY[((long)b * Co + co) * P + p0 + pp] : 0.f;
        }
        for (int e = threadIdx.x; e < Ci * kWgChunk; e += blockDim.x) {
            const int ci = e / kWgChunk, pp = e % kWgChunk;
            xs[ci][pp] = p0 + pp < P ? ld(X, ((long)b * Ci + ci) * P + p0 + pp) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int o = threadIdx.x + 256 * j;
            if (o < nout) {
                const int co = o / (Ci + 1), ci = o % (Ci + 1);
                float a = 0.f;
                if (ci < Ci) {
                    for (int pp = 0; pp < kWgChunk; ++pp) a += ys[co][pp] * xs[ci][pp];
                } else {
                    for (int pp = 0; pp < kWgChunk; ++pp) a += ys[co][pp];
                }
                acc[j] += a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int o = threadIdx.x + 256 * j;
        if (o < nout) {
            const int co = o / (Ci + 1), ci = o % (Ci + 1);
            atomicAdd(ci < Ci ? &dW[co * Ci + ci] : &db[co], acc[j]);
        }
    }
}

inline unsigned wgrad_grid(long P, int B) {
    const long n = (long)B * ((P + kWgChunk - 1) / kWgChunk);
    return (unsigned)(n < 1216 ? n : 1216);
}

// ------------------------------------------------------- tensor-core GEMMs
// In the BF16 storage mode the three contractions that dominate the network
// run on the tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulation in tensor memory): the x transform (rows x NX against the
// twiddle table), the layer output (per (b, y) row: x against [v ; basis],
// transposed so the 128 x positions are the MMA's M), and the weight
// gradients (sum over pixels of dY X^T).  BF16 activations are exact BF16
// operands; FP32 operands (twiddles, basis, weights, spectra, cotangents)
// are split into hi + lo BF16 parts and the products hi.hi + hi.lo + lo.hi
// are accumulated, which keeps about 16 bits of each, well above the BF16
// storage of the activations.  Tiles: M = 128 rows, K in chunks of 64
// (16 per instruction), operands staged by the block's threads in the
// canonical K-major layout; one thread issues the MMAs, the block waits on
// the commit with a bounded poll and reads the accumulator with tcgen05.ld.
// A wait that gives up raises g_fno_status (read back by the synchronising
// FNO calls) and the block frees its tensor memory and returns.
constexpr int kTcM = 128, kTcKC = 64;
constexpr long kFnoWaitLimit = 1L << 22;
__device__ int g_fno_status;

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// 8 BF16 values as one 16-byte word
__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&v)[8]) {
    uint4 r;
    r.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
    r.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
    r.z = (uint32_t)__bfloat16_as_ushort(v[4]) | ((uint32_t)__bfloat16_as_ushort(v[5]) << 16);
    r.w = (uint32_t)__bfloat16_as_ushort(v[6]) | ((uint32_t)__bfloat16_as_ushort(v[7]) << 16);
    return r;
}

// twiddle operand of the tensor-core x transform: chunk c, part (hi, lo),
// row n = 2 kx + (0: Re, 1: Im) of e^{-2 pi i kx x / NX}, column x - 64 c;
// rows n >= 2M are zero
__global__ void k_init_xbimg(unsigned char* __restrict__ img, int NX, int M, int NP) {
    const long total = (long)(NX / kTcKC) * NP * kTcKC;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / (NP * kTcKC)), e = (int)(idx % (NP * kTcKC));
        const int n = e / kTcKC, k = e % kTcKC;
        const int x = c * kTcKC + k, kx = n >> 1;
        double v = 0.0;
        if (n < 2 * M) {
            double sn, cs;
            sincospi(2.0 * (double)(((long)kx * x) % NX) / (double)NX, &sn, &cs);
            v = (n & 1) ? -sn : cs;
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
        const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
        unsigned char* base = img + (long)c * 2 * NP * kTcKC * 2;
        const int o = tc5::kmajor_off<2>(n, k, kTcKC);
        *reinterpret_cast<__nv_bfloat16*>(base + o) = hi;
        *reinterpret_cast<__nv_bfloat16*>(base + NP * kTcKC * 2 + o) = lo;
    }
}

// A[row][kx] = scale(kx) sum_x X[row][x] e^{-2 pi i kx x / NX} on the tensor
// cores; NX a multiple of 64, one block per 128 rows, NP = 2M rounded up
// to 16.  SI = BF16 (activations, exact) or float (cotangents, split).
template <typename SI, int NP>
__global__ void __launch_bounds__(128) k_dft_x_tc(const SI* __restrict__ X, float2* __restrict__ A,
                                                  const unsigned char* __restrict__ bimg, long rows, int NX, int M,
                                                  float scale0, float scale1) {
    constexpr bool SPLIT = std::is_same<SI, float>::value;
    constexpr int A_BYTES = kTcM * kTcKC * 2, B_BYTES = NP * kTcKC * 2;
    constexpr uint32_t NCOL = NP <= 32 ? 32 : 64;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + A_BYTES;
    unsigned char* b_hi = smem + 2 * A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_hi + 2 * B_BYTES);
    uint32_t* slot = reinterpret_cast<uint32_t*>(b_hi + 2 * B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    if (warp == 0) tc5::tmem_alloc(slot, NCOL);
    if (tid == 0) tc5::mbar_init(mb, 1);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = *slot;
    const long r0 = (long)blockIdx.x * kTcM;
    const int nch = NX / kTcKC;
    uint32_t phase = 0;
    bool ok = true;
    for (int c = 0; c < nch && ok; ++c) {
        for (int e = tid; e < kTcM * 8; e += blockDim.x) {
            const int r = e >> 3, ch = e & 7;
            const long row = r0 + r;
            const int o = tc5::kmajor_off<2>(r, ch * 8, kTcKC);
            if constexpr (SPLIT) {
                float f[8];
                if (row < rows) {
                    const float4 f0 = *reinterpret_cast<const float4*>(X + row * NX + c * kTcKC + ch * 8);
                    const float4 f1 = *reinterpret_cast<const float4*>(X + row * NX + c * kTcKC + ch * 8 + 4);
                    f[0] = f0.x; f[1] = f0.y; f[2] = f0.z; f[3] = f0.w;
                    f[4] = f1.x; f[5] = f1.y; f[6] = f1.z; f[7] = f1.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[i] = 0.f;
                }
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) split_bf16(f[i], hi[i], lo[i]);
                *reinterpret_cast<uint4*>(a_hi + o) = pack8(hi);
                *reinterpret_cast<uint4*>(a_lo + o) = pack8(lo);
            } else {
                const uint4 w = row < rows ? *reinterpret_cast<const uint4*>(X + row * NX + c * kTcKC + ch * 8)
                                           : make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(a_hi + o) = w;
            }
        }
        {
            const uint4* src = reinterpret_cast<const uint4*>(bimg + (long)c * 2 * B_BYTES);
            uint4* dst = reinterpret_cast<uint4*>(b_hi);
            for (int e = tid; e < 2 * B_BYTES / 16; e += blockDim.x) dst[e] = src[e];
        }
        tc5::fence_async_smem();
        tc5::fence_before_sync();
        __syncthreads();
        tc5::fence_after_sync();
        if (tid == 0) {
            constexpr uint32_t id = tc5::idesc(false, kTcM, NP);
            constexpr uint32_t sbo = (kTcKC / 8) * 128;
            const uint32_t ah = (uint32_t)__cvta_generic_to_shared(a_hi), al = (uint32_t)__cvta_generic_to_shared(a_lo);
            const uint32_t bh = (uint32_t)__cvta_generic_to_shared(b_hi), bl = bh + B_BYTES;
#pragma unroll
            for (int kc = 0; kc < kTcKC / 16; ++kc) {
                const uint64_t dah = tc5::smem_desc(ah + kc * 256, 128, sbo);
                const uint64_t dbh = tc5::smem_desc(bh + kc * 256, 128, sbo);
                tc5::mma_bf16(tmem, dah, dbh, id, (c > 0 || kc > 0) ? 1u : 0u);
                tc5::mma_bf16(tmem, dah, tc5::smem_desc(bl + kc * 256, 128, sbo), id, 1u);
                if constexpr (SPLIT) tc5::mma_bf16(tmem, tc5::smem_desc(al + kc * 256, 128, sbo), dbh, id, 1u);
            }
            tc5::commit(mb);
        }
        const bool got = tc5::mbar_wait(mb, phase, kFnoWaitLimit);
        phase ^= 1u;
        tc5::fence_after_sync();
        ok = __syncthreads_and(got) != 0;       // the same decision in every thread
    }
    if (ok) {
        const long row = r0 + tid;
#pragma unroll
        for (int cc = 0; cc < NP / 16; ++cc) {
            float v[16];
            tc5::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cc * 16, v);
            if (row < rows) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int kx = cc * 8 + j;
                    if (kx < M) {
                        const float sc = kx == 0 ? scale0 : scale1;
                        A[row * M + kx] = make_float2(v[2 * j] * sc, v[2 * j + 1] * sc);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicCAS(&g_fno_status, 0, (int)MM_ERR_TIMEOUT);
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc5::tmem_free(tmem, NCOL);
}

// layer output on the tensor cores for one (b, y) row and 128 x positions
// (NX a multiple of 128), the transposed form of k_layer_out's GEMM:
//   a[co][x] = bias[co] + sum_k Aop[x][k] Bop[co][k],
//   Aop = [v rows ; basis rows]^T (K = W + 2M padded to KP, a multiple of 16),
//   Bop = [W | Re U, Im U],
// then v_next = GELU(a) (or a for the last layer).  N = 32 (rows co >= W zero).
__global__ void __launch_bounds__(128) k_layer_out_tc(const __nv_bfloat16* __restrict__ v, const float2* __restrict__ U,
                                                      const float* __restrict__ Wt, const float* __restrict__ bias,
                                                      const float* __restrict__ basis, __nv_bfloat16* __restrict__ a_out,
                                                      __nv_bfloat16* __restrict__ v_next, int W, int NY, int NX, int M,
                                                      int KP, int last) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int A_BYTES = kTcM * KP * 2, B_BYTES = 32 * KP * 2;
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + A_BYTES;
    unsigned char* b_hi = smem + 2 * A_BYTES;
    unsigned char* b_lo = b_hi + B_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + B_BYTES);
    uint32_t* slot = reinterpret_cast<uint32_t*>(b_lo + B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int y = blockIdx.x, b = blockIdx.y, x0 = blockIdx.z * kTcM;
    const long P = (long)NY * NX;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    if (warp == 0) tc5::tmem_alloc(slot, 32);
    if (tid == 0) tc5::mbar_init(mb, 1);
    // A: thread tid owns row x = x0 + tid
    {
        const int x = x0 + tid;
        for (int k8 = 0; k8 < KP; k8 += 8) {
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = k8 + i;
                if (k < W) {
                    hi[i] = v[((long)b * W + k) * P + (long)y * NX + x];
                    lo[i] = __float2bfloat16_rn(0.f);
                } else if (k < W + 2 * M) {
                    split_bf16(basis[(long)(k - W) * NX + x], hi[i], lo[i]);
                } else {
                    hi[i] = lo[i] = __float2bfloat16_rn(0.f);
                }
            }
            const int o = tc5::kmajor_off<2>(tid, k8, KP);
            *reinterpret_cast<uint4*>(a_hi + o) = pack8(hi);
            *reinterpret_cast<uint4*>(a_lo + o) = pack8(lo);
        }
    }
    // B: [co][k], 32 rows
    for (int e = tid; e < 32 * (KP / 8); e += blockDim.x) {
        const int co = e / (KP / 8), k8 = (e % (KP / 8)) * 8;
        __nv_bfloat16 hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = k8 + i;
            float val = 0.f;
            if (co < W) {
                if (k < W) {
                    val = Wt[co * W + k];
                } else if (k < W + 2 * M) {
                    const float2 u = U[(((long)b * W + co) * NY + y) * M + ((k - W) >> 1)];
                    val = ((k - W) & 1) ? u.y : u.x;
                }
            }
            split_bf16(val, hi[i], lo[i]);
        }
        const int o = tc5::kmajor_off<2>(co, k8, KP);
        *reinterpret_cast<uint4*>(b_hi + o) = pack8(hi);
        *reinterpret_cast<uint4*>(b_lo + o) = pack8(lo);
    }
    tc5::fence_async_smem();
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = *slot;
    if (tid == 0) {
        const uint32_t id = tc5::idesc(false, kTcM, 32);
        const uint32_t sbo = (uint32_t)(KP / 8) * 128;
        const uint32_t ah = (uint32_t)__cvta_generic_to_shared(a_hi), al = (uint32_t)__cvta_generic_to_shared(a_lo);
        const uint32_t bh = (uint32_t)__cvta_generic_to_shared(b_hi), bl = (uint32_t)__cvta_generic_to_shared(b_lo);
        for (int kc = 0; kc < KP / 16; ++kc) {
            const uint64_t dah = tc5::smem_desc(ah + kc * 256, 128, sbo), dbh = tc5::smem_desc(bh + kc * 256, 128, sbo);
            tc5::mma_bf16(tmem, dah, dbh, id, kc > 0 ? 1u : 0u);
            tc5::mma_bf16(tmem, dah, tc5::smem_desc(bl + kc * 256, 128, sbo), id, 1u);
            tc5::mma_bf16(tmem, tc5::smem_desc(al + kc * 256, 128, sbo), dbh, id, 1u);
        }
        tc5::commit(mb);
    }
    const bool got = tc5::mbar_wait(mb, 0, kFnoWaitLimit);
    tc5::fence_after_sync();
    const bool ok = __syncthreads_and(got) != 0;
    if (ok) {
        const int x = x0 + tid;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            float d[16];
            tc5::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cc * 16, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int co = cc * 16 + j;
                if (co < W) {
                    const float val = d[j] + bias[co];
                    const long o = ((long)b * W + co) * P + (long)y * NX + x;
                    a_out[o] = __float2bfloat16_rn(val);
                    v_next[o] = __float2bfloat16_rn(last ? val : gelu(val));
                }
            }
        }
    } else if (tid == 0) {
        atomicCAS(&g_fno_status, 0, (int)MM_ERR_TIMEOUT);
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc5::tmem_free(tmem, 32);
}

inline size_t layer_out_tc_smem(int KP) { return (size_t)2 * kTcM * KP * 2 + (size_t)2 * 32 * KP * 2 + 64; }

// dW[co][ci] += sum_{b,p} dY[b][co][p] X[b][ci][p], db[co] += sum dY, on the
// tensor cores: M = 128 rows of which the first Co (<= 32) are dY's
// channels (split hi + lo), N = NP >= Ci + 1 columns of X's channels plus a
// column of ones (the bias), K = 64 pixels per step; blocks walk the
// pixel chunks of all samples (P a multiple of 64) and add their sums once.
template <typename SX, int NP>
__global__ void __launch_bounds__(128) k_wgrad_tc(const float* __restrict__ dY, const SX* __restrict__ X,
                                                  float* __restrict__ dW, float* __restrict__ db, int Co, int Ci,
                                                  long P, int B) {
    constexpr bool SPLITX = std::is_same<SX, float>::value;
    constexpr int A_BYTES = kTcM * kTcKC * 2, B_BYTES = NP * kTcKC * 2;
    constexpr uint32_t NCOL = NP <= 32 ? 32 : 64;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + A_BYTES;
    unsigned char* b_hi = smem + 2 * A_BYTES;
    unsigned char* b_lo = b_hi + B_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + B_BYTES);
    uint32_t* slot = reinterpret_cast<uint32_t*>(b_lo + B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    if (warp == 0) tc5::tmem_alloc(slot, NCOL);
    if (tid == 0) tc5::mbar_init(mb, 1);
    // zero both operands once: rows co >= Co of A and columns beyond Ci of B
    // stay zero, the bias column is set below
    for (int e = tid; e < (2 * A_BYTES + 2 * B_BYTES) / 16; e += blockDim.x)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int e = tid; e < kTcKC; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(b_hi + tc5::kmajor_off<2>(Ci, e, kTcKC)) = __float2bfloat16_rn(1.f);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = *slot;
    const long cps = P / kTcKC;
    uint32_t phase = 0;
    bool ok = true, any = false;
    for (long c = blockIdx.x; c < (long)B * cps && ok; c += gridDim.x) {
        const int b = (int)(c / cps);
        const long p0 = (c % cps) * kTcKC;
        for (int e = tid; e < Co * 8; e += blockDim.x) {
            const int co = e >> 3, ch = e & 7;
            const float* src = dY + ((long)b * Co + co) * P + p0 + ch * 8;
            const float4 f0 = *reinterpret_cast<const float4*>(src), f1 = *reinterpret_cast<const float4*>(src + 4);
            const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) split_bf16(f[i], hi[i], lo[i]);
            const int o = tc5::kmajor_off<2>(co, ch * 8, kTcKC);
            *reinterpret_cast<uint4*>(a_hi + o) = pack8(hi);
            *reinterpret_cast<uint4*>(a_lo + o) = pack8(lo);
        }
        for (int e = tid; e < Ci * 8; e += blockDim.x) {
            const int ci = e >> 3, ch = e & 7;
            const int o = tc5::kmajor_off<2>(ci, ch * 8, kTcKC);
            if constexpr (SPLITX) {
                const float* src = X + ((long)b * Ci + ci) * P + p0 + ch * 8;
                const float4 f0 = *reinterpret_cast<const float4*>(src), f1 = *reinterpret_cast<const float4*>(src + 4);
                const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) split_bf16(f[i], hi[i], lo[i]);
                *reinterpret_cast<uint4*>(b_hi + o) = pack8(hi);
                *reinterpret_cast<uint4*>(b_lo + o) = pack8(lo);
            } else {
                *reinterpret_cast<uint4*>(b_hi + o) =
                    *reinterpret_cast<const uint4*>(X + ((long)b * Ci + ci) * P + p0 + ch * 8);
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before_sync();
        __syncthreads();
        tc5::fence_after_sync();
        if (tid == 0) {
            constexpr uint32_t id = tc5::idesc(false, kTcM, NP);
            constexpr uint32_t sbo = (kTcKC / 8) * 128;
            const uint32_t ah = (uint32_t)__cvta_generic_to_shared(a_hi), al = (uint32_t)__cvta_generic_to_shared(a_lo);
            const uint32_t bh = (uint32_t)__cvta_generic_to_shared(b_hi), bl = (uint32_t)__cvta_generic_to_shared(b_lo);
#pragma unroll
            for (int kc = 0; kc < kTcKC / 16; ++kc) {
                const uint64_t dbh = tc5::smem_desc(bh + kc * 256, 128, sbo);
                const uint64_t dah = tc5::smem_desc(ah + kc * 256, 128, sbo);
                tc5::mma_bf16(tmem, dah, dbh, id, (any || kc > 0) ? 1u : 0u);
                tc5::mma_bf16(tmem, tc5::smem_desc(al + kc * 256, 128, sbo), dbh, id, 1u);
                if constexpr (SPLITX) tc5::mma_bf16(tmem, dah, tc5::smem_desc(bl + kc * 256, 128, sbo), id, 1u);
            }
            tc5::commit(mb);
        }
        any = true;
        const bool got = tc5::mbar_wait(mb, phase, kFnoWaitLimit);
        phase ^= 1u;
        tc5::fence_after_sync();
        ok = __syncthreads_and(got) != 0;
    }
    if (ok && any && warp == 0) {
#pragma unroll
        for (int cc = 0; cc < NP / 16; ++cc) {
            float d[16];
            tc5::tmem_ld16(tmem + cc * 16, d);
            const int co = tid;
            if (co < Co) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int ci = cc * 16 + j;
                    if (ci < Ci) atomicAdd(&dW[co * Ci + ci], d[j]);
                    else if (ci == Ci) atomicAdd(&db[co], d[j]);
                }
            }
        }
    } else if (!ok && tid == 0) {
        atomicCAS(&g_fno_status, 0, (int)MM_ERR_TIMEOUT);
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc5::tmem_free(tmem, NCOL);
}

template <int NP> constexpr size_t gemm_tc_smem() { return (size_t)2 * kTcM * kTcKC * 2 + (size_t)2 * NP * kTcKC * 2 + 64; }

// per-sample sums of (h - t)^2 and t^2
__global__ void k_loss_sums(const float* __restrict__ h, const float* __restrict__ t, double* __restrict__ red, long n) {
    const int b = blockIdx.y;
    __shared__ double r1[256], r2[256];
    double s1 = 0, s2 = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double d = (double)h[b * n + i] - t[b * n + i];
        s1 += d * d;
        s2 += (double)t[b * n + i] * t[b * n + i];
    }
    r1[threadIdx.x] = s1;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            r1[threadIdx.x] += r1[threadIdx.x + k];
            r2[threadIdx.x] += r2[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&red[2 * b], r1[0]);
        atomicAdd(&red[2 * b + 1], r2[0]);
    }
}

// dh = 2 (h - t) / (B sum t^2)
__global__ void k_loss_grad(const float* __restrict__ h, const float* __restrict__ t, const double* __restrict__ red,
                            float* __restrict__ dh, long n, int B) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * n) return;
    const int b = (int)(i / n);
    dh[i] = (float)(2.0 * ((double)h[i] - t[i]) / (B * red[2 * b + 1]));
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// inverse-x basis rows for k_layer_out: [2 kx] = c_kx cos / P, [2 kx + 1] = c_kx (-sin) / P
__global__ void k_init_basis(const float2* twx, float* basis, int NX, int NY, int M) {
    const double invP = 1.0 / ((double)NX * NY);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * M * NX; i += gridDim.x * blockDim.x) {
        const int r = i / NX, x = i % NX, kx = r >> 1;
        const float2 w = twx[(long)kx * NX + x];
        const double c = (kx == 0 ? 1.0 : 2.0) * invP;
        basis[i] = (float)(c * ((r & 1) ? w.y : w.x));
    }
}

__global__ void k_init_tw(float2* twx, float2* twy, int NX, int NY, int M) {
    const int total = M * NX + 2 * M * NY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        double s, c;
        if (i < M * NX) {
            const int kx = i / NX, x = i % NX;
            sincospi(-2.0 * (double)((long)kx * x % NX) / NX, &s, &c);
            twx[i] = make_float2((float)c, (float)s);
        } else {
            const int j = i - M * NX;
            const int r = j / NY, y = j % NY;
            const int ky = ky_of(r, M, NY);
            sincospi(-2.0 * (double)((long)ky * y % NY) / NY, &s, &c);
            twy[j] = make_float2((float)c, (float)s);
        }
    }
}

constexpr int kFT = 256;
inline unsigned g1(long n) { return (unsigned)((n + kFT - 1) / kFT); }

int ffail(mm_fno* f, int code, const char* msg) {
    if (f) f->err = msg;
    return fail(nullptr, code, "%s", msg);
}

inline int round16(int v) { return (v + 15) / 16 * 16; }

// after a synchronisation: TIMEOUT if a tensor-core wait gave up since the
// last check (the flag is cleared), else OK
int tc_status(mm_fno* f) {
    int st = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&st, g_fno_status, sizeof(int));
    if (e != cudaSuccess) return ffail(f, MM_ERR_CUDA, cudaGetErrorString(e));
    if (st) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_fno_status, &zero, sizeof(int));
        return ffail(f, st, "a tensor-core wait of the FNO kernels gave up (TIMEOUT)");
    }
    return MM_OK;
}

// x transform rows x NX -> A (tensor cores when the operand image exists)
template <typename SI>
void dft_x(mm_fno* f, const SI* X, float2* out, long rows, float scale0, float scale1) {
    if (f->xbimg) {
        const unsigned g = (unsigned)((rows + kTcM - 1) / kTcM);
        switch (f->xNP) {
            case 16: k_dft_x_tc<SI, 16><<<g, 128, gemm_tc_smem<16>(), f->stream>>>(X, out, f->xbimg, rows, f->nx, f->M, scale0, scale1); return;
            case 32: k_dft_x_tc<SI, 32><<<g, 128, gemm_tc_smem<32>(), f->stream>>>(X, out, f->xbimg, rows, f->nx, f->M, scale0, scale1); return;
            case 48: k_dft_x_tc<SI, 48><<<g, 128, gemm_tc_smem<48>(), f->stream>>>(X, out, f->xbimg, rows, f->nx, f->M, scale0, scale1); return;
            default: k_dft_x_tc<SI, 64><<<g, 128, gemm_tc_smem<64>(), f->stream>>>(X, out, f->xbimg, rows, f->nx, f->M, scale0, scale1); return;
        }
    }
    k_dft_x<SI><<<(unsigned)((rows + kDxRows - 1) / kDxRows), 256, 0, f->stream>>>(X, out, f->twx, rows, f->nx, f->M,
                                                                                  scale0, scale1);
}

// weight gradients of a 1x1 map (tensor cores in the BF16 mode when the
// pixel count is a multiple of 64)
template <typename SX>
void wgrad(mm_fno* f, const float* dY, const SX* X, float* dW, float* db, int Co, int Ci, int B) {
    const long P = f->P;
    if (f->store_bf16 && P % kTcKC == 0) {
        const long chunks = (long)B * (P / kTcKC);
        const unsigned g = (unsigned)(chunks < 608 ? chunks : 608);
        if (round16(Ci + 1) <= 16)
            k_wgrad_tc<SX, 16><<<g, 128, gemm_tc_smem<16>(), f->stream>>>(dY, X, dW, db, Co, Ci, P, B);
        else if (round16(Ci + 1) <= 32)
            k_wgrad_tc<SX, 32><<<g, 128, gemm_tc_smem<32>(), f->stream>>>(dY, X, dW, db, Co, Ci, P, B);
        else
            k_wgrad_tc<SX, 48><<<g, 128, gemm_tc_smem<48>(), f->stream>>>(dY, X, dW, db, Co, Ci, P, B);
        return;
    }
    k_wgrad<SX><<<wgrad_grid(P, B), 256, 0, f->stream>>>(dY, X, dW, db, Co, Ci, P, B);
}

#define FNO_CHECK(f)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess) return ffail((f), MM_ERR_CUDA, cudaGetErrorString(e_));         \
    } while (0)

template <typename SS> int forward_t(mm_fno* f, const float* m, float* h, int B) {
    const long P = f->P;
    const int W = f->W, NX = f->nx, NY = f->ny, M = f->M, K = f->K;
    SS* v = (SS*)f->v;
    SS* a = (SS*)f->a;
    const long vs = (long)f->max_batch * W * P;
    k_chan<float, SS><<<g1((long)B * P), kFT, 0, f->stream>>>(m, f->params + f->o_P, f->params + f->o_p, v, 3, W, P, B,
                                                              1.f, 0);
    FNO_CHECK(f);
    for (int l = 0; l < f->L; ++l) {
        SS* vl = v + l * vs;
        float2* S = f->S + (long)l * f->max_batch * W * K;
        dft_x<SS>(f, vl, f->A, (long)B * W * NY, 1.f, 1.f);
        k_dft_y_modes<<<g1(8L * B * W * 2 * M * M), kFT, 0, f->stream>>>(f->A, S, f->twy, B * W, NY, M, -1.f);
        k_mix<<<g1((long)B * W * K), kFT, 0, f->stream>>>(S, (const float2*)(f->params + f->o_R[l]), f->T, B, W, K, 0);
        k_dft_y<<<g1((long)B * W * NY * M), kFT, 0, f->stream>>>(f->T, f->U, f->twy, B * W, NY, M, 0, 1.f);
        if constexpr (std::is_same<SS, __nv_bfloat16>::value) {
            if (NX % kTcM == 0) {
                const int KP = round16(W + 2 * M);
                k_layer_out_tc<<<dim3((unsigned)NY, (unsigned)B, (unsigned)(NX / kTcM)), 128, layer_out_tc_smem(KP),
                                 f->stream>>>(vl, f->U, f->params + f->o_W[l], f->params + f->o_b[l], f->basis,
                                              a + l * vs, v + (l + 1) * vs, W, NY, NX, M, KP, l == f->L - 1);
                FNO_CHECK(f);
                continue;
            }
        }
        k_layer_out<SS><<<dim3((unsigned)NY, (unsigned)B, (unsigned)((NX + kLoTile - 1) / kLoTile)), 256,
                          layer_out_smem(W, M), f->stream>>>(vl, f->U, f->params + f->o_W[l], f->params + f->o_b[l],
                                                             f->basis, a + l * vs, v + (l + 1) * vs, B, W, NY, NX, M,
                                                             l == f->L - 1);
        FNO_CHECK(f);
    }
    k_chan<SS, float><<<g1((long)B * P), kFT, 0, f->stream>>>(v + f->L * vs, f->params + f->o_Q, f->params + f->o_q, h, W,
                                                              3, P, B, f->out_scale, 0);
    FNO_CHECK(f);
    return MM_OK;
}

template <typename SS> int backward_t(mm_fno* f, const float* dh, int B) {
    const long P = f->P;
    const int W = f->W, NX = f->nx, NY = f->ny, M = f->M, K = f->K;
    SS* v = (SS*)f->v;
    SS* a = (SS*)f->a;
    const long vs = (long)f->max_batch * W * P;
    float* dv = (float*)f->dv;
    float* dv2 = dv + vs;
    float* G = f->grads;
    // projection: dQ += dh v_L^T, dq += sum dh, dv_L = Q^T dh
    wgrad<SS>(f, dh, v + f->L * vs, G + f->o_Q, G + f->o_q, 3, W, B);
    k_chan<float, float><<<g1((long)B * P), kFT, 0, f->stream>>>(dh, f->params + f->o_Q, nullptr, dv, 3, W, P, B, 1.f, 1);
    FNO_CHECK(f);
    for (int l = f->L - 1; l >= 0; --l) {
        SS* vl = v + l * vs;
        float2* S = f->S + (long)l * f->max_batch * W * K;
        // da = dv * GELU'(a)
        k_gelu_bwd<SS><<<g1((long)B * W * P), kFT, 0, f->stream>>>(dv, a + l * vs, (long)B * W * P, l == f->L - 1);
        // channel part
        wgrad<SS>(f, dv, vl, G + f->o_W[l], G + f->o_b[l], W, W, B);
        k_chan<float, float><<<g1((long)B * P), kFT, 0, f->stream>>>(dv, f->params + f->o_W[l], nullptr, dv2, W, W, P, B,
                                                                     1.f, 1);
        // spectral part: dU = c / P sum_x da e^{-i theta}
        dft_x<float>(f, dv, f->U, (long)B * W * NY, 1.f / (float)P, 2.f / (float)P);
        k_dft_y_modes<<<g1(8L * B * W * 2 * M * M), kFT, 0, f->stream>>>(f->U, f->T, f->twy, B * W, NY, M, -1.f);
        k_mix_grad<<<g1((long)W * W * K), kFT, 0, f->stream>>>(f->T, S, (float2*)(G + f->o_R[l]), B, W, K);
        // dS = R^H dT into U (free again; the stored spectra S stay intact for a later backward)
        k_mix<<<g1((long)B * W * K), kFT, 0, f->stream>>>(f->T, (const float2*)(f->params + f->o_R[l]), f->U, B, W, K, 1);
        k_dft_y<<<g1((long)B * W * NY * M), kFT, 0, f->stream>>>(f->U, f->A, f->twy, B * W, NY, M, 0, 1.f);
        k_dft_x_adj<<<g1((long)B * W * NY * NX), kFT, 0, f->stream>>>(f->A, dv2, f->twx, (long)B * W * NY, NX, M, 1);
        FNO_CHECK(f);
        std::swap(dv, dv2);
    }
    return MM_OK;
}

}  // namespace

void fno_grid(const mm_fno* f, int* nx, int* ny) {
    *nx = f->nx;
    *ny = f->ny;
}

cudaStream_t fno_swap_stream(mm_fno* f, cudaStream_t s) {
    cudaStream_t old = f->stream;
    f->stream = s;
    return old;
}

}  // namespace mm

using namespace mm;

extern "C" {

int mm_fno_create(mm_fno** out, int nx, int ny, int width, int modes, int layers, int store_bf16, int max_batch,
                  unsigned long long seed, void* stream) {
    if (!out) return fail(nullptr, MM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2 || width < 1 || width > 32 || modes < 1 || modes > kMaxModes || 2 * modes > ny ||
        modes > nx / 2 || layers < 1 ||
        max_batch < 1)
        return fail(nullptr, MM_ERR_INVALID_ARG, "FNO sizes: width <= 32, modes <= 32, 2 modes <= ny, modes <= nx / 2");
    mm_fno* f = new mm_fno();
    f->nx = nx;
    f->ny = ny;
    f->W = width;
    f->M = modes;
    f->L = layers;
    f->store_bf16 = store_bf16 ? 1 : 0;
    f->max_batch = max_batch;
    f->stream = (cudaStream_t)stream;
    f->P = (long)nx * ny;
    f->MY = 2 * modes;
    f->K = f->MY * modes;
    f->out_scale = 1.f;
    int dev = 0;
    cudaError_t ce = stream ? cudaStreamGetDevice(f->stream, &dev) : cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaSetDevice(dev);
    f->device = dev;
    // parameter layout
    long o = 0;
    f->o_P = o; o += 3L * width;
    f->o_p = o; o += width;
    for (int l = 0; l < layers; ++l) {
        f->o_W.push_back(o); o += (long)width * width;
        f->o_b.push_back(o); o += width;
        f->o_R.push_back(o); o += 2L * width * width * f->K;
    }
    f->o_Q = o; o += 3L * width;
    f->o_q = o; o += 3;
    f->nparams = o;
    const size_t es = f->store_bf16 ? 2 : 4;
    const long vs = (long)max_batch * width * f->P;
    bool ok = ce == cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
    };
    A((void**)&f->params, o * 4);
    A((void**)&f->grads, o * 4);
    A((void**)&f->adam_m, o * 4);
    A((void**)&f->adam_v, o * 4);
    A(&f->v, (size_t)(layers + 1) * vs * es);
    A(&f->a, (size_t)layers * vs * es);
    A((void**)&f->S, (size_t)layers * max_batch * width * f->K * sizeof(float2));
    A((void**)&f->A, (size_t)max_batch * width * ny * modes * sizeof(float2));
    A((void**)&f->T, (size_t)max_batch * width * f->K * sizeof(float2));
    A((void**)&f->U, (size_t)max_batch * width * ny * modes * sizeof(float2));
    A(&f->dv, 2 * (size_t)vs * 4);
    A((void**)&f->twx, (size_t)modes * nx * sizeof(float2));
    A((void**)&f->twy, (size_t)2 * modes * ny * sizeof(float2));
    A((void**)&f->basis, (size_t)2 * modes * nx * sizeof(float));
    A((void**)&f->red, (size_t)2 * max_batch * sizeof(double));
    f->xNP = (2 * modes + 15) / 16 * 16;
    if (f->store_bf16 && nx % kTcKC == 0) A((void**)&f->xbimg, (size_t)(nx / kTcKC) * 2 * f->xNP * kTcKC * 2);
    if (!ok) {
        cudaGetLastError();
        mm_fno_destroy(f);
        return fail(nullptr, MM_ERR_NOMEM, "FNO allocation failed");
    }
    // initialisation: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for 1x1 maps,
    // spectral weights uniform * 1/(W W), biases 0 (seeded host generator)
    std::vector<float> h(o, 0.f);
    unsigned long long s = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto rnd = [&]() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return ((double)(s >> 11) / 9007199254740992.0) * 2.0 - 1.0;
    };
    for (long i = 0; i < 3L * width; ++i) h[f->o_P + i] = (float)(rnd() / std::sqrt(3.0));
    for (int l = 0; l < layers; ++l) {
        for (long i = 0; i < (long)width * width; ++i) h[f->o_W[l] + i] = (float)(rnd() / std::sqrt((double)width));
        for (long i = 0; i < 2L * width * width * f->K; ++i) h[f->o_R[l] + i] = (float)(rnd() / ((double)width * width));
    }
    for (long i = 0; i < 3L * width; ++i) h[f->o_Q + i] = (float)(rnd() / std::sqrt((double)width));
    ce = cudaMemcpy(f->params, h.data(), o * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(f->grads, 0, o * 4);
    if (ce == cudaSuccess) ce = cudaMemset(f->adam_m, 0, o * 4);
    if (ce == cudaSuccess) ce = cudaMemset(f->adam_v, 0, o * 4);
    k_init_tw<<<64, 256, 0, f->stream>>>(f->twx, f->twy, nx, ny, modes);
    k_init_basis<<<64, 256, 0, f->stream>>>(f->twx, f->basis, nx, ny, modes);
    if (f->xbimg) k_init_xbimg<<<64, 256, 0, f->stream>>>(f->xbimg, nx, modes, f->xNP);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(k_layer_out_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)layer_out_tc_smem(round16(32 + 2 * kMaxModes)));
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(k_dft_x_tc<__nv_bfloat16, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)gemm_tc_smem<64>());
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(k_dft_x_tc<float, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)gemm_tc_smem<64>());
    // the layer-output GEMM keeps its K x 256 operand in dynamic shared memory
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(k_layer_out<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)layer_out_smem(32, kMaxModes));
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(k_layer_out<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)layer_out_smem(32, kMaxModes));
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(f->stream);
    if (ce != cudaSuccess) {
        mm_fno_destroy(f);
        return fail(nullptr, MM_ERR_CUDA, "FNO setup: %s", cudaGetErrorString(ce));
    }
    *out = f;
    return MM_OK;
}

void mm_fno_destroy(mm_fno* f) {
    if (!f) return;
    cudaSetDevice(f->device);
    cudaStreamSynchronize(f->stream);
    void* ptrs[] = {f->params, f->grads, f->adam_m, f->adam_v, f->v,   f->a,     f->S,  f->A,
                    f->T,      f->U,     f->dv,     f->twx,    f->twy, f->basis, f->red, f->xbimg};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete f;
}

long mm_fno_num_params(const mm_fno* f) { return f ? f->nparams : 0; }

int mm_fno_forward(mm_fno* f, const void* m, void* h, int batch) {
    if (!f || !m || !h || batch < 1 || batch > f->max_batch) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_fno_forward: bad arguments");
    if (cudaSetDevice(f->device) != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "cudaSetDevice");
    return f->store_bf16 ? forward_t<__nv_bfloat16>(f, (const float*)m, (float*)h, batch)
                         : forward_t<float>(f, (const float*)m, (float*)h, batch);
}

int mm_fno_backward(mm_fno* f, const void* m, const void* dh, int batch) {
    if (!f || !m || !dh || batch < 1 || batch > f->max_batch) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_fno_backward: bad arguments");
    if (f->out_scale != 1.f) return ffail(f, MM_ERR_INVALID_ARG, "mm_fno_backward: output scale must be 1 while training");
    if (cudaSetDevice(f->device) != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "cudaSetDevice");
    int rc = f->store_bf16 ? backward_t<__nv_bfloat16>(f, (const float*)dh, batch) : backward_t<float>(f, (const float*)dh, batch);
    if (rc) return rc;
    // lift: dP += dv_0 m^T, dp += sum dv_0 (dv_0 ends in the buffer the last swap selected)
    const long vs = (long)f->max_batch * f->W * f->P;
    float* dv0 = (float*)f->dv + ((f->L % 2) ? vs : 0);
    wgrad<float>(f, dv0, (const float*)m, f->grads + f->o_P, f->grads + f->o_p, f->W, 3, batch);
    FNO_CHECK(f);
    return MM_OK;
}

int mm_fno_zero_grad(mm_fno* f) {
    if (!f) return fail(nullptr, MM_ERR_INVALID_ARG, "fno is NULL");
    cudaSetDevice(f->device);
    cudaError_t e = cudaMemsetAsync(f->grads, 0, f->nparams * 4, f->stream);
    return e == cudaSuccess ? MM_OK : ffail(f, MM_ERR_CUDA, cudaGetErrorString(e));
}

int mm_fno_adam_step(mm_fno* f, double lr, double beta1, double beta2, double eps, long step) {
    if (!f || step < 1) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_fno_adam_step: bad arguments");
    cudaSetDevice(f->device);
    const float c1 = (float)(1.0 - std::pow(beta1, (double)step)), c2 = (float)(1.0 - std::pow(beta2, (double)step));
    k_adam<<<g1(f->nparams), kFT, 0, f->stream>>>(f->params, f->grads, f->adam_m, f->adam_v, f->nparams, (float)lr,
                                                  (float)beta1, (float)beta2, (float)eps, c1, c2);
    FNO_CHECK(f);
    return MM_OK;
}

int mm_fno_loss(mm_fno* f, const void* h, const void* target, void* dh, int batch, double* loss_out) {
    if (!f || !h || !target || batch < 1 || batch > f->max_batch) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_fno_loss: bad arguments");
    cudaSetDevice(f->device);
    const long n = 3 * f->P;
    cudaError_t e = cudaMemsetAsync(f->red, 0, 2 * batch * sizeof(double), f->stream);
    if (e != cudaSuccess) return ffail(f, MM_ERR_CUDA, cudaGetErrorString(e));
    dim3 g(64, batch);
    k_loss_sums<<<g, 256, 0, f->stream>>>((const float*)h, (const float*)target, f->red, n);
    if (dh) k_loss_grad<<<g1(batch * n), kFT, 0, f->stream>>>((const float*)h, (const float*)target, f->red, (float*)dh, n, batch);
    FNO_CHECK(f);
    if (loss_out) {
        std::vector<double> r(2 * batch);
        e = cudaMemcpyAsync(r.data(), f->red, 2 * batch * sizeof(double), cudaMemcpyDeviceToHost, f->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
        if (e != cudaSuccess) return ffail(f, MM_ERR_CUDA, cudaGetErrorString(e));
        int rc = tc_status(f);
        if (rc) return rc;
        double L = 0;
        for (int b = 0; b < batch; ++b) L += r[2 * b] / r[2 * b + 1];
        *loss_out = L / batch;
    }
    return MM_OK;
}

int mm_fno_params(mm_fno* f, float* host_params, float* host_grads, const float* host_set) {
    if (!f) return fail(nullptr, MM_ERR_INVALID_ARG, "fno is NULL");
    cudaSetDevice(f->device);
    cudaError_t e = cudaStreamSynchronize(f->stream);
    if (e == cudaSuccess) {
        int rc = tc_status(f);
        if (rc) return rc;
    }
    if (e == cudaSuccess && host_set) e = cudaMemcpy(f->params, host_set, f->nparams * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && host_params) e = cudaMemcpy(host_params, f->params, f->nparams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_grads) e = cudaMemcpy(host_grads, f->grads, f->nparams * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MM_OK : ffail(f, MM_ERR_CUDA, cudaGetErrorString(e));
}

int mm_fno_set_output_scale(mm_fno* f, double scale) {
    if (!f) return fail(nullptr, MM_ERR_INVALID_ARG, "fno is NULL");
    f->out_scale = (float)scale;
    return MM_OK;
}

}  // extern "C"
