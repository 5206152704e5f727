// Tensor-core split-precision DFT stages (5th-generation tensor cores,
// tcgen05 with the accumulator in tensor memory).
//
// A batch of 32-point complex DFTs is one real GEMM: the 128 lines of a tile
// are the rows of A (interleaved re/im, K = 64), B is the real form of the
// 32 x 32 DFT matrix (N = 64 outputs: Re X_k = sum c x.re - s x.im,
// Im X_k = sum s x.re + c x.im with c + i s = exp(dir 2 pi i n k / 32)).
// FP32 operands are split into hi + lo parts of the tensor-core type
// (TF32: round to 10 mantissa bits; BF16: round to 7) and the product is
// formed as hi.hi + hi.lo + lo.hi with FP32 accumulation, which keeps
// about twice the operand type's bits.  One elected thread issues the MMAs
// (operands in shared memory, canonical K-major layout without swizzle),
// tcgen05.commit signals an mbarrier, every warp reads its 32 accumulator
// rows back with tcgen05.ld.  Every wait is bounded: on a timeout the block
// raises the library's device status and frees its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "mm_regfft.cuh"

namespace mm {
namespace {

constexpr int kTcLines = 128;    // M: lines per tile
constexpr int kTcK = 64;         // K: 32 complex inputs
constexpr int kTcN = 64;         // N: 32 complex outputs
constexpr long kTcWaitLimit = 1L << 22;

// DFT matrix of each mode and direction in the GEMM's B layout
// ([N][K] values, hi and lo parts), built once per device
__device__ float g_dft_f32[2][2][kTcN * kTcK];            // [dir][hi/lo]
__device__ __nv_bfloat16 g_dft_bf16[2][2][kTcN * kTcK];
// the same matrices as shared-memory images (K-major canonical layout, hi
// then lo), copied into a block with 16-byte loads
__device__ __align__(16) unsigned char g_bimg_tf32[2][2 * kTcN * kTcK * 4];
__device__ __align__(16) unsigned char g_bimg_bf16[2][2 * kTcN * kTcK * 2];
// BF16 in three parts (hi, mid, lo) for the y passes: about 24 bits
__device__ __align__(16) unsigned char g_bimg_bf16x3[2][3 * kTcN * kTcK * 2];
__device__ int g_tc_status;

bool g_tables_ready[64] = {false};
std::mutex g_tables_mutex;

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__global__ void k_init_dft_tables() {
    for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < 2 * kTcN * kTcK; idx += blockDim.x * gridDim.x) {
        const int d = idx / (kTcN * kTcK), e = idx % (kTcN * kTcK);
        const int j = e / kTcK, kk = e % kTcK;        // output j (2k + part), input kk (2n + part)
        const int k = j >> 1, n = kk >> 1;
        const double dir = d == 0 ? -1.0 : 1.0;
        double c, s;
        sincospi(dir * 2.0 * (double)((n * k) % 32) / 32.0, &s, &c);
        double v;
        if ((j & 1) == 0) v = (kk & 1) == 0 ? c : -s;   // Re X_k
        else v = (kk & 1) == 0 ? s : c;                  // Im X_k
        const float hi32 = tf32_round((float)v);
        g_dft_f32[d][0][e] = hi32;
        g_dft_f32[d][1][e] = tf32_round((float)(v - (double)hi32));
        const __nv_bfloat16 hb = __float2bfloat16_rn((float)v);
        g_dft_bf16[d][0][e] = hb;
        g_dft_bf16[d][1][e] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hb)));
    }
}

template <int ES> __device__ __forceinline__ int kmajor_off(int r, int k, int K);

__global__ void k_init_dft_images() {
    for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < 2 * kTcN * kTcK; idx += blockDim.x * gridDim.x) {
        const int d = idx / (kTcN * kTcK), e = idx % (kTcN * kTcK);
        const int j = e / kTcK, kk = e % kTcK;
        const int o4 = kmajor_off<4>(j, kk, kTcK), o2 = kmajor_off<2>(j, kk, kTcK);
        *reinterpret_cast<float*>(&g_bimg_tf32[d][o4]) = g_dft_f32[d][0][e];
        *reinterpret_cast<float*>(&g_bimg_tf32[d][kTcN * kTcK * 4 + o4]) = g_dft_f32[d][1][e];
        *reinterpret_cast<__nv_bfloat16*>(&g_bimg_bf16[d][o2]) = g_dft_bf16[d][0][e];
        *reinterpret_cast<__nv_bfloat16*>(&g_bimg_bf16[d][kTcN * kTcK * 2 + o2]) = g_dft_bf16[d][1][e];
        {
            const int j = e / kTcK, kk = e % kTcK;
            const int k = j >> 1, n = kk >> 1;
            double sn, cs;
            sincospi((d == 0 ? -1.0 : 1.0) * 2.0 * (double)((n * k) % 32) / 32.0, &sn, &cs);
            const double v = (j & 1) == 0 ? ((kk & 1) == 0 ? cs : -sn) : ((kk & 1) == 0 ? sn : cs);
            const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
            const double r1 = v - (double)__bfloat162float(h);
            const __nv_bfloat16 mid = __float2bfloat16_rn((float)r1);
            const __nv_bfloat16 lo = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(mid)));
            *reinterpret_cast<__nv_bfloat16*>(&g_bimg_bf16x3[d][o2]) = h;
            *reinterpret_cast<__nv_bfloat16*>(&g_bimg_bf16x3[d][kTcN * kTcK * 2 + o2]) = mid;
            *reinterpret_cast<__nv_bfloat16*>(&g_bimg_bf16x3[d][2 * kTcN * kTcK * 2 + o2]) = lo;
        }
    }
}

// byte offset of element (r, k) in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, adjacent in K (LBO = 128 B), row
// groups SBO = (K / elements per 16 B) * 128 B apart
template <int ES> __device__ __forceinline__ int kmajor_off(int r, int k, int K) {
    constexpr int KC = 16 / ES;
    return (r >> 3) * ((K / KC) * 128) + (k / KC) * 128 + (r & 7) * 16 + (k % KC) * ES;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::tf32 or kind::f16 (bf16) instruction descriptor: D f32, K-major A and B
template <bool TF32> __device__ __forceinline__ uint32_t instr_desc() {
    const uint32_t fmt = TF32 ? 2u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcLines >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (TF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long limit = kTcWaitLimit) {
    for (long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Self-test of the bounded wait: the block initialises an mbarrier that
// expects one arrival nobody makes and polls it `limit` times; the wait gives
// up, raises TIMEOUT in the device status and the block returns.
__global__ void k_wait_selftest(long limit, int* gave_up) {
    __shared__ uint64_t bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
    __syncthreads();
    const bool ok = mbar_wait(a, 0, limit);
    if (!ok && threadIdx.x == 0) {
        atomicCAS(&g_tc_status, 0, (int)MM_ERR_TIMEOUT);
        *gave_up = 1;
    }
}

// Shared memory of one tile: A hi/lo [128 x 64], B hi/lo [64 x 64] (element
// size ES), the mbarrier and the tensor-memory address.
template <int ES, int PARTS = 2> struct TcSmem {
    static constexpr int A_BYTES = kTcLines * kTcK * ES;
    static constexpr int B_BYTES = kTcN * kTcK * ES;
    static constexpr int BYTES = PARTS * A_BYTES + PARTS * B_BYTES + 64;
};

// Batched 32-point DFT of `nlines` contiguous lines of 32 float2 values.
template <bool TF32>
__global__ void __launch_bounds__(kTcLines) k_dft32_tc(const float2* __restrict__ in, float2* __restrict__ out,
                                                       long nlines, int dir_index) {
    constexpr int ES = TF32 ? 4 : 2;
    using S = TcSmem<ES>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + S::A_BYTES;
    unsigned char* b_hi = smem + 2 * S::A_BYTES;
    unsigned char* b_lo = b_hi + S::B_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + S::B_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_lo + S::B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tmem_slot)),
                     "r"(kTcN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a));

    // B: the DFT matrix, [N][K] in the K-major layout
    for (int e = tid; e < kTcN * kTcK; e += blockDim.x) {
        const int j = e / kTcK, kk = e % kTcK;
        const int o = kmajor_off<ES>(j, kk, kTcK);
        if constexpr (TF32) {
            *reinterpret_cast<float*>(b_hi + o) = g_dft_f32[dir_index][0][e];
            *reinterpret_cast<float*>(b_lo + o) = g_dft_f32[dir_index][1][e];
        } else {
            *reinterpret_cast<__nv_bfloat16*>(b_hi + o) = g_dft_bf16[dir_index][0][e];
            *reinterpret_cast<__nv_bfloat16*>(b_lo + o) = g_dft_bf16[dir_index][1][e];
        }
    }
    // A: one line per thread, split into hi + lo
    const long line = (long)blockIdx.x * kTcLines + tid;
    for (int n = 0; n < 32; ++n) {
        float2 v = line < nlines ? in[line * 32 + n] : make_float2(0.f, 0.f);
        const float xs[2] = {v.x, v.y};
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const int o = kmajor_off<ES>(tid, 2 * n + part, kTcK);
            const float x = xs[part];
            if constexpr (TF32) {
                const float h = tf32_round(x);
                *reinterpret_cast<float*>(a_hi + o) = h;
                *reinterpret_cast<float*>(a_lo + o) = tf32_round(x - h);
            } else {
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                *reinterpret_cast<__nv_bfloat16*>(a_hi + o) = h;
                *reinterpret_cast<__nv_bfloat16*>(a_lo + o) = __float2bfloat16_rn(x - __bfloat162float(h));
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        const uint32_t idesc = instr_desc<TF32>();
        const uint32_t sbo_a = (kTcK / (16 / ES)) * 128, sbo_b = sbo_a;
        const uint32_t A[2] = {(uint32_t)__cvta_generic_to_shared(a_hi), (uint32_t)__cvta_generic_to_shared(a_lo)};
        const uint32_t Bm[2] = {(uint32_t)__cvta_generic_to_shared(b_hi), (uint32_t)__cvta_generic_to_shared(b_lo)};
        // hi.hi + hi.lo + lo.hi
        const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
        constexpr int KMMA = TF32 ? 8 : 16;          // K per instruction: 32 bytes = 2 core matrices
        uint32_t acc = 0;
        for (int p = 0; p < 3; ++p) {
            for (int kc = 0; kc < kTcK / KMMA; ++kc) {
                const uint64_t ad = smem_desc(A[pa[p]] + kc * 256, 128, sbo_a);
                const uint64_t bd = smem_desc(Bm[pb[p]] + kc * 256, 128, sbo_b);
                mma<TF32>(tmem, ad, bd, idesc, acc);
                acc = 1;
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                     : "memory");
    }
    const bool ok = mbar_wait(mbar_a, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if ((tid & 31) == 0) atomicCAS(&g_tc_status, 0, (int)MM_ERR_TIMEOUT);
    } else {
        uint32_t r[64];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
            "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
            "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
              "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
              "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
              "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
              "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (line < nlines) {
#pragma unroll
            for (int k = 0; k < 32; ++k) out[line * 32 + k] = make_float2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}

// Four-step column transform of length L = 32 L2 for B = 128 / L2 adjacent
// columns, persistent over tiles (B columns of one plane each): level 1
// (rows (t2, b), 32-point DFT over n1 of x[t2 + L2 n1]) is one tensor-core
// GEMM of the 128 rows; on read-back each row is twiddled by w_L^(t2 k1) and
// transposed through shared memory; level 2 (thread (k1, b), L2-point DFT
// over n2 in registers) writes X[k1 + 32 k2].  The DFT-matrix operand and
// the tensor memory are set up once per block; the line operands are split
// into parts of the tensor-core type and stored 16 bytes at a time: TF32 hi +
// lo (products hi.hi + hi.lo + lo.hi, about 21 bits), BF16 hi + mid + lo
// (products hi.hi + hi.mid + mid.hi + mid.mid + hi.lo + lo.hi; the dropped
// ones are below 2^-23 relative, so about 24 bits, the FP32 path's own
// precision).  PIN: the upper half of the input rows is zero (K = 32 real
// inputs); POUT: only the lower half of the output rows is written.
template <int L2, int DIR, bool PIN, bool POUT, bool TF32>
__global__ void __launch_bounds__(32 * (128 / L2))
    k_cols_tc(const float2* in, float2* out, int Hx, ColGeom cg, const float2* __restrict__ tw, int ntx,
              long ntiles) {
    constexpr int B = 128 / L2, L = 32 * L2;
    constexpr int ES = TF32 ? 4 : 2;
    constexpr int PARTS = TF32 ? 2 : 3;
    constexpr int KA = PIN ? 32 : 64;
    constexpr int EPV = 16 / ES;                            // elements per 16-byte store
    using S = TcSmem<ES, PARTS>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + S::A_BYTES;
    unsigned char* a_mid = smem + 2 * S::A_BYTES;           // BF16 only
    unsigned char* b_hi = smem + PARTS * S::A_BYTES;
    unsigned char* b_part[3] = {b_hi, b_hi + S::B_BYTES, b_hi + 2 * S::B_BYTES};   // BF16: hi, mid, lo
    unsigned char* b_lo = TF32 ? b_part[1] : b_part[2];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_hi + PARTS * S::B_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_hi + PARTS * S::B_BYTES + 16);
    float2* T = reinterpret_cast<float2*>(smem);            // level-2 transpose, reuses A after the MMA
    static_assert(L * B * 8 <= PARTS * S::A_BYTES, "transpose must fit in the A operand space");
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = B < 16 ? 16 / B - 1 : 0;
    const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(mbar);
    const int dir_index = DIR < 0 ? 0 : 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tmem_slot)),
                     "r"(kTcN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a));
    {
        // B (TF32: hi, lo; BF16: hi, mid, lo): one image copy
        const uint4* src = reinterpret_cast<const uint4*>(TF32 ? g_bimg_tf32[dir_index] : g_bimg_bf16x3[dir_index]);
        uint4* dst = reinterpret_cast<uint4*>(b_hi);
        for (int e = tid; e < PARTS * S::B_BYTES / 16; e += blockDim.x) dst[e] = src[e];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int t2 = tid / B, bb = tid % B;
    uint32_t phase = 0;
    bool ok = true;
    for (long it = blockIdx.x; it < ntiles; it += gridDim.x, phase ^= 1u) {
        const int col0 = (int)(it % ntx) * B;
        const int p = (int)(it / ntx);
        const int pi = p % cg.n_inner, po = p / cg.n_inner;
        const float2* ib = in + pi * cg.in_inner + po * cg.in_outer;
        float2* ob = out + pi * cg.out_inner + po * cg.out_outer;
        const bool act = col0 + bb < Hx;
        if (tid < kTcLines) {
            float2 v[KA / 2];
#pragma unroll
            for (int n1 = 0; n1 < KA / 2; ++n1)
                v[n1] = act ? ib[(long)(t2 + L2 * n1) * cg.rs_in + col0 + bb] : make_float2(0.f, 0.f);
            // operand row tid: element kk = 2 n1 + part; EPV consecutive elements per 16-byte store
#pragma unroll
            for (int c = 0; c < KA / EPV; ++c) {
                float xs[EPV];
#pragma unroll
                for (int q = 0; q < EPV; ++q) {
                    const float2 z = v[(c * EPV + q) >> 1];
                    xs[q] = (q & 1) ? z.y : z.x;
                }
                const int o = kmajor_off<ES>(tid, c * EPV, kTcK);
                if constexpr (TF32) {
                    float h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        h[q] = tf32_round(xs[q]);
                        l[q] = tf32_round(xs[q] - h[q]);
                    }
                    *reinterpret_cast<float4*>(a_hi + o) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(a_lo + o) = make_float4(l[0], l[1], l[2], l[3]);
                } else {
                    uint32_t hw[4], mw[4], lw[4];   // element q at byte 2 q of the 16-byte slot
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        __nv_bfloat16 hh[2], mm[2], ll[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const float x = xs[2 * q + u];
                            hh[u] = __float2bfloat16_rn(x);
                            const float r1 = x - __bfloat162float(hh[u]);      // exact
                            mm[u] = __float2bfloat16_rn(r1);
                            ll[u] = __float2bfloat16_rn(r1 - __bfloat162float(mm[u]));
                        }
                        const __nv_bfloat162 hp = __halves2bfloat162(hh[0], hh[1]);
                        const __nv_bfloat162 mp = __halves2bfloat162(mm[0], mm[1]);
                        const __nv_bfloat162 lp = __halves2bfloat162(ll[0], ll[1]);
                        hw[q] = *reinterpret_cast<const uint32_t*>(&hp);
                        mw[q] = *reinterpret_cast<const uint32_t*>(&mp);
                        lw[q] = *reinterpret_cast<const uint32_t*>(&lp);
                    }
                    *reinterpret_cast<uint4*>(a_hi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(a_mid + o) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
                    *reinterpret_cast<uint4*>(a_lo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t idesc = instr_desc<TF32>();
            const uint32_t sbo = (kTcK / (16 / ES)) * 128;
            // parts: 0 hi, 1 lo, 2 mid (BF16)
            const uint32_t A[3] = {(uint32_t)__cvta_generic_to_shared(a_hi), (uint32_t)__cvta_generic_to_shared(a_lo),
                                   (uint32_t)__cvta_generic_to_shared(a_mid)};
            const uint32_t Bm[3] = {(uint32_t)__cvta_generic_to_shared(b_hi), (uint32_t)__cvta_generic_to_shared(b_lo),
                                    (uint32_t)__cvta_generic_to_shared(b_part[1])};
            // TF32: hi.hi, hi.lo, lo.hi; BF16 adds hi.mid, mid.hi, mid.mid
            constexpr int NPROD = TF32 ? 3 : 6;
            const int pa[6] = {0, 0, 1, 0, 2, 2}, pb[6] = {0, 1, 0, 2, 0, 2};
            constexpr int KMMA = TF32 ? 8 : 16;
            uint32_t acc = 0;
            for (int q = 0; q < NPROD; ++q)
                for (int kc = 0; kc < KA / KMMA; ++kc) {
                    mma<TF32>(tmem, smem_desc(A[pa[q]] + kc * 256, 128, sbo), smem_desc(Bm[pb[q]] + kc * 256, 128, sbo),
                              idesc, acc);
                    acc = 1;
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                         : "memory");
        }
        ok = mbar_wait(mbar_a, phase);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        if (tid < kTcLines) {
            uint32_t r[64];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
                "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
                "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                  "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                  "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
                  "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
                  "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
                  "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
                  "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // all MMA reads of A are complete (mbarrier), so T may overwrite A
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                float2 y = make_float2(__uint_as_float(r[2 * k1]), __uint_as_float(r[2 * k1 + 1]));
                if (k1 > 0) {
                    float2 w = tw[t2 * k1];
                    if (DIR > 0) w.y = -w.y;
                    y = cmul(y, w);
                }
                T[((k1 * L2) + (t2 ^ (k1 & m))) * B + bb] = y;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        {
            const int k1 = tid / B, b2 = tid % B;
            const bool act2 = col0 + b2 < Hx;
            float2 u[L2];
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) u[n2] = T[((k1 * L2) + (n2 ^ (k1 & m))) * B + b2];
            dif<L2, DIR, false>(u);
            constexpr int NOUT = POUT ? L2 / 2 : L2;
            if (act2) {
#pragma unroll
                for (int k2 = 0; k2 < NOUT; ++k2) ob[(long)(k1 + 32 * k2) * cg.rs_out + col0 + b2] = u[dif_pos<L2>(k2)];
            }
        }
        __syncthreads();   // T (the A space) is free for the next tile
    }
    if (!ok) {
        if ((tid & 31) == 0) atomicCAS(&g_tc_status, 0, (int)MM_ERR_TIMEOUT);
        mbar_wait(mbar_a, phase);   // let an MMA still in flight finish before the memory goes (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}

template <int L2, int DIR, bool TF32>
int launch_cols_tc(mm_ctx* ctx, const float2* in, float2* out, int nplanes, ColGeom g, const float2* tw) {
    constexpr int B = 128 / L2;
    const int bytes = TF32 ? TcSmem<4, 2>::BYTES : TcSmem<2, 3>::BYTES;
    auto fn = k_cols_tc<L2, DIR, (DIR < 0), (DIR > 0), TF32>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return fail(ctx, MM_ERR_CUDA, "tensor-core pass setup: %s", cudaGetErrorString(e));
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * B, bytes);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess || per_sm < 1) return fail(ctx, MM_ERR_CUDA, "tensor-core pass: no resident block");
    const int ntx = (ctx->Hx + B - 1) / B;
    const long ntiles = (long)ntx * nplanes;
    // tiles per block (measured): two for the 128-thread L = 1024 pass (one:
    // more operand staging per line; more: less overlap); the 256-thread
    // L = 512 pass runs persistent, one block per resident slot
    const long grid = L2 == 32 ? (ntiles + 1) / 2 : std::min<long>(ntiles, (long)per_sm * sms);
    fn<<<(unsigned)grid, 32 * B, bytes, ctx->stream>>>(in, out, ctx->Hx, g, tw, ntx, ntiles);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int ensure_tables(int dev, cudaStream_t st) {
    if (dev < 0 || dev >= 64) return fail(nullptr, MM_ERR_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_tables_mutex);
    if (!g_tables_ready[dev]) {
        k_init_dft_tables<<<16, 256, 0, st>>>();
        k_init_dft_images<<<16, 256, 0, st>>>();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "DFT table setup: %s", cudaGetErrorString(e));
        g_tables_ready[dev] = true;
    }
    return MM_OK;
}

}  // namespace

int tc_prepare(mm_ctx* ctx) { return ensure_tables(ctx->device, ctx->stream); }

int tc_cols(mm_ctx* ctx, const float2* in, float2* out, int L, int dir, int nplanes, ColGeom g, const float2* tw) {
    const bool tf32 = ctx->fft_mode == MM_TC_TF32;
    if (L == 512) {
        if (dir < 0) return tf32 ? launch_cols_tc<16, -1, true>(ctx, in, out, nplanes, g, tw)
                                 : launch_cols_tc<16, -1, false>(ctx, in, out, nplanes, g, tw);
        return tf32 ? launch_cols_tc<16, 1, true>(ctx, in, out, nplanes, g, tw)
                    : launch_cols_tc<16, 1, false>(ctx, in, out, nplanes, g, tw);
    }
    if (dir < 0) return tf32 ? launch_cols_tc<32, -1, true>(ctx, in, out, nplanes, g, tw)
                             : launch_cols_tc<32, -1, false>(ctx, in, out, nplanes, g, tw);
    return tf32 ? launch_cols_tc<32, 1, true>(ctx, in, out, nplanes, g, tw)
                : launch_cols_tc<32, 1, false>(ctx, in, out, nplanes, g, tw);
}

}  // namespace mm

using namespace mm;

extern "C" int mm_set_fft_mode(mm_ctx* ctx, int mode) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (mode != 0 && mode != MM_TC_TF32 && mode != MM_TC_BF16 && mode != MM_FFT_FF && mode != MM_FFT_F4)
        return fail(ctx, MM_ERR_INVALID_ARG, "bad FFT mode %d", mode);
    if (mode == MM_FFT_F4) {
        if (!f4_supported(ctx))
            return fail(ctx, MM_ERR_INVALID_ARG, "the fused y-z-y pass needs an MM_F32 context with ny = 512, nz = 16");
        MM_BIND(ctx);
        int rc = f4_prepare(ctx);
        if (rc) return rc;
        ctx->fft_mode = mode;
        return MM_OK;
    }
    if (mode == MM_FFT_FF) {
        auto p2 = [](int n) { return n > 0 && (n & (n - 1)) == 0; };
        if (ctx->prec != MM_F64) return fail(ctx, MM_ERR_INVALID_ARG, "float-float passes need an MM_F64 context");
        if (!p2(ctx->Px) || !p2(ctx->Py) || !p2(ctx->Pz))
            return fail(ctx, MM_ERR_INVALID_ARG, "float-float passes need power-of-two padded sizes (nx, ny, nz)");
        MM_BIND(ctx);
        int rc = demag_prepare_ff(ctx);
        if (rc) return rc;
        ctx->fft_mode = mode;
        return MM_OK;
    }
    if (mode != 0 && ctx->prec != MM_F32) return fail(ctx, MM_ERR_INVALID_ARG, "tensor-core passes need an MM_F32 context");
    MM_BIND(ctx);
    if (mode != 0) {
        int rc = tc_prepare(ctx);
        if (rc) return fail(ctx, rc, "%s", mm_last_error(nullptr));
    }
    ctx->fft_mode = mode;
    return MM_OK;
}

extern "C" int mm_tc_status(mm_ctx* ctx) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    int status = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&status, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, MM_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (status) return fail(ctx, status, "a tensor-core wait timed out");
    return MM_OK;
}

extern "C" int mm_tc_wait_selftest(long limit, void* stream) {
    if (limit < 1 || limit > (1L << 20)) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_tc_wait_selftest: limit in 1..2^20");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = st ? cudaStreamGetDevice(st, &dev) : cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    int* flag = nullptr;
    int gave_up = 0, status = 0;
    const int zero = 0;
    if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, st>>>(limit, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&gave_up, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&status, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    // clear the status again: the self-test leaves the library usable
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (flag) cudaFree(flag);
    if (e != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "mm_tc_wait_selftest: %s", cudaGetErrorString(e));
    if (gave_up && status == MM_ERR_TIMEOUT) return fail(nullptr, MM_ERR_TIMEOUT, "bounded wait gave up as intended");
    return MM_OK;
}

extern "C" int mm_dft32_tc(const void* in, void* out, long nlines, int mode, int direction, void* stream) {
    if (!in || !out || nlines < 0) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_dft32_tc: bad arguments");
    if (mode != MM_TC_TF32 && mode != MM_TC_BF16) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_dft32_tc: bad mode");
    if (direction != -1 && direction != 1) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_dft32_tc: direction is -1 or 1");
    if (nlines == 0) return MM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = st ? cudaStreamGetDevice(st, &dev) : cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "mm_dft32_tc: %s", cudaGetErrorString(e));
    int rc = ensure_tables(dev, st);
    if (rc) return rc;
    const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    const unsigned grid = (unsigned)((nlines + kTcLines - 1) / kTcLines);
    const int dir_index = direction < 0 ? 0 : 1;
    if (e == cudaSuccess) {
        if (mode == MM_TC_TF32) {
            const int bytes = TcSmem<4>::BYTES;
            e = cudaFuncSetAttribute(k_dft32_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e == cudaSuccess) k_dft32_tc<true><<<grid, kTcLines, bytes, st>>>((const float2*)in, (float2*)out, nlines, dir_index);
        } else {
            const int bytes = TcSmem<2>::BYTES;
            e = cudaFuncSetAttribute(k_dft32_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e == cudaSuccess) k_dft32_tc<false><<<grid, kTcLines, bytes, st>>>((const float2*)in, (float2*)out, nlines, dir_index);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&status, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "mm_dft32_tc: %s", cudaGetErrorString(e));
    if (status) return fail(nullptr, status, "mm_dft32_tc: tensor-core wait timed out");
    return MM_OK;
}
