// Standalone field evaluations (mm_exchange_field, mm_effective_field) for
// FP32 contexts with uniform material, nx a multiple of 4 and no DMI: four
// x-consecutive cells per thread with 16-byte loads and stores, the exchange
// part of the fused stage kernel on its own.
//   H_ex,i = (2 A / (mu0 Ms)) sum_axis sum_nb (m_nb - m_i) / d_axis^2 (Eq. 2,
//   read for unit m, free boundary: a missing neighbour adds nothing);
//   effective: H_ex + anisotropy + Zeeman + the caller's demag field.
// Other contexts keep the generic one-cell-per-thread kernel.
#include "mm_fields.cuh"

namespace mm {
namespace {

struct Quad {
    float4 x, y, z;
};

__device__ __forceinline__ float4 ld4q(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4q(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& el(float4& v, int j) { return (&v.x)[j]; }
__device__ __forceinline__ float el(const float4& v, int j) { return (&v.x)[j]; }

__device__ __forceinline__ Quad ld_quad(const float* a, long i, long N) {
    return {ld4q(a + i), ld4q(a + i + N), ld4q(a + i + 2 * N)};
}
// acc += w (nb - c), component-wise over the four cells
__device__ __forceinline__ void acc_diff(Quad& acc, const Quad& nb, const Quad& c, float w) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        el(acc.x, j) += w * (el(nb.x, j) - el(c.x, j));
        el(acc.y, j) += w * (el(nb.y, j) - el(c.y, j));
        el(acc.z, j) += w * (el(nb.z, j) - el(c.z, j));
    }
}

// MODE 0: exchange only; MODE 1: exchange + anisotropy + Zeeman + Hd
template <int MODE>
__global__ void __launch_bounds__(256) k_field4(Params<float> p, float wx, float wy, float wz,
                                                const float* __restrict__ m, const float* __restrict__ Hd,
                                                float* __restrict__ H) {
    const long i = 4 * ((long)blockIdx.x * blockDim.x + threadIdx.x);
    const long N = p.N;
    if (i >= N) return;
    int x, y, z;
    decompose(i, p.nx, p.ny, x, y, z);
    const Quad c = ld_quad(m, i, N);
    Quad h = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
    Quad xl, xr;
    xl.x = make_float4(x > 0 ? m[i - 1] : c.x.x, c.x.x, c.x.y, c.x.z);
    xl.y = make_float4(x > 0 ? m[i - 1 + N] : c.y.x, c.y.x, c.y.y, c.y.z);
    xl.z = make_float4(x > 0 ? m[i - 1 + 2 * N] : c.z.x, c.z.x, c.z.y, c.z.z);
    const bool rx = x + 4 < p.nx;
    xr.x = make_float4(c.x.y, c.x.z, c.x.w, rx ? m[i + 4] : c.x.w);
    xr.y = make_float4(c.y.y, c.y.z, c.y.w, rx ? m[i + 4 + N] : c.y.w);
    xr.z = make_float4(c.z.y, c.z.z, c.z.w, rx ? m[i + 4 + 2 * N] : c.z.w);
    acc_diff(h, xl, c, wx);
    acc_diff(h, xr, c, wx);
    const long sy = p.nx, sz = (long)p.nx * p.ny;
    if (y > 0) acc_diff(h, ld_quad(m, i - sy, N), c, wy);
    if (y < p.ny - 1) acc_diff(h, ld_quad(m, i + sy, N), c, wy);
    if (z > 0) acc_diff(h, ld_quad(m, i - sz, N), c, wz);
    if (z < p.nz - 1) acc_diff(h, ld_quad(m, i + sz, N), c, wz);
    if constexpr (MODE == 1) {
        const Quad d = ld_quad(Hd, i, N);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const V3<float> mi = {el(c.x, j), el(c.y, j), el(c.z, j)};
            const V3<float> l = local_at(p, mi, p.Ms);
            el(h.x, j) += l.x + el(d.x, j);
            el(h.y, j) += l.y + el(d.y, j);
            el(h.z, j) += l.z + el(d.z, j);
        }
    }
    st4q(H + i, h.x);
    st4q(H + i + N, h.y);
    st4q(H + i + 2 * N, h.z);
}

}  // namespace

// MM_OK with *done = true when the four-cell kernel ran; *done = false
// leaves the call to the generic kernel
int field4(mm_ctx* ctx, const void* m, const void* Hd, void* H, bool effective, bool* done) {
    *done = false;
    if (ctx->prec != MM_F32 || ctx->has_Ms_cell || ctx->has_A_cell || ctx->Ms == 0.0 || ctx->nx % 4 != 0 ||
        ctx->dmi_type != 0)
        return MM_OK;
    // 16-byte accesses: every component plane of every array must be aligned
    const uintptr_t mask = (uintptr_t)m | (uintptr_t)H | (effective ? (uintptr_t)Hd : 0);
    if (mask % 16 != 0 || ctx->N % 4 != 0) return MM_OK;
    KernelTimer kt(ctx, MM_K_REDUCE);
    const Params<float> p = make_params<float>(ctx);
    const float inv = 1.f / p.Ms;
    const long quads = ctx->N / 4;
    const unsigned blocks = (unsigned)((quads + 255) / 256);
    if (effective)
        k_field4<1><<<blocks, 256, 0, ctx->stream>>>(p, p.A * p.cx * inv, p.A * p.cy * inv, p.A * p.cz * inv,
                                                     (const float*)m, (const float*)Hd, (float*)H);
    else
        k_field4<0><<<blocks, 256, 0, ctx->stream>>>(p, p.A * p.cx * inv, p.A * p.cy * inv, p.A * p.cz * inv,
                                                     (const float*)m, nullptr, (float*)H);
    *done = true;
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace mm
