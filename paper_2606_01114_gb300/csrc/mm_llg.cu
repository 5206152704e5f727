// Local part of the effective field and the LLG time step (paper,
// Implementation section, Eq. 1 and Eq. 2; RKF45 paragraph).
//
//   exchange (Eq. 2, unit m):  H_i = 2 / (mu0 Ms_i) sum_nb A_h (m_nb - m_i) / d^2,
//       A_h = 2 A_i A_nb / (A_i + A_nb), free boundary, Ms = 0 cells are
//       vacuum (no field, skipped as neighbours);
//   anisotropy  H = 2 Ku / (mu0 Ms) (m.u) u,   Zeeman H = H_ext;
//   LLG (Eq. 1, unit m):  dm/dt = -gamma / (1 + alpha^2) [m x H + alpha m x (m x H)].
//
// K7 (k_stage) fuses, for one Runge-Kutta stage, the exchange stencil, the
// local fields, the sum with the demag field of the stage state, the LLG
// right-hand side and the stage sum of the next trial state, in one pass
// over HBM.  Its last-stage instance also forms the new state
// (4th-order solution for RKF45), the embedded error max |m5 - m4| (block
// reduction + one atomic max per block) and the renormalisation.  The RKF45
// step control (k_controller) runs on the device, so a step needs no host
// synchronisation.  Energies and the torque maximum (K9) accumulate in FP64.
#include <cmath>

#include "mm_ff.cuh"
#include "mm_fields.cuh"

namespace mm {
namespace {

// ---------------------------------------------------- Butcher tableaux
// classic RK4 and Fehlberg's RKF45 (4th-order weights propagated)
__host__ __device__ constexpr double rk_a(int method, int i, int j) {
    if (method == MM_RK4) {
        if (i == 1 && j == 0) return 0.5;
        if (i == 2 && j == 1) return 0.5;
        if (i == 3 && j == 2) return 1.0;
        return 0.0;
    }
    switch (i * 8 + j) {
        case 1 * 8 + 0: return 1.0 / 4.0;
        case 2 * 8 + 0: return 3.0 / 32.0;
        case 2 * 8 + 1: return 9.0 / 32.0;
        case 3 * 8 + 0: return 1932.0 / 2197.0;
        case 3 * 8 + 1: return -7200.0 / 2197.0;
        case 3 * 8 + 2: return 7296.0 / 2197.0;
        case 4 * 8 + 0: return 439.0 / 216.0;
        case 4 * 8 + 1: return -8.0;
        case 4 * 8 + 2: return 3680.0 / 513.0;
        case 4 * 8 + 3: return -845.0 / 4104.0;
        case 5 * 8 + 0: return -8.0 / 27.0;
        case 5 * 8 + 1: return 2.0;
        case 5 * 8 + 2: return -3544.0 / 2565.0;
        case 5 * 8 + 3: return 1859.0 / 4104.0;
        case 5 * 8 + 4: return -11.0 / 40.0;
        default: return 0.0;
    }
}
__host__ __device__ constexpr double rk_b(int method, int j) {
    if (method == MM_RK4) {
        return j == 0 ? 1.0 / 6.0 : j == 1 ? 1.0 / 3.0 : j == 2 ? 1.0 / 3.0 : j == 3 ? 1.0 / 6.0 : 0.0;
    }
    return j == 0 ? 25.0 / 216.0 : j == 2 ? 1408.0 / 2565.0 : j == 3 ? 2197.0 / 4104.0 : j == 4 ? -1.0 / 5.0 : 0.0;
}
// b5 - b4 (RKF45 error weights)
__host__ __device__ constexpr double rk_e(int method, int j) {
    if (method == MM_RK4) return 0.0;
    constexpr double b5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
    return b5[j] - rk_b(method, j);
}
__host__ __device__ constexpr int rk_stages(int method) { return method == MM_RK4 ? 4 : 6; }

// block-wide max of a non-negative double, then one atomicMax of its bits
__device__ __forceinline__ void block_max_atomic(double v, unsigned long long* target) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0 && v > 0.0) atomicMax(target, (unsigned long long)__double_as_longlong(v));
    }
}

__device__ __forceinline__ void block_sum_atomic(double v, double* target) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(target, v);
    }
}

// Block reductions of per-thread values of the path's type T: the warp
// stage runs in T (FP32 adds for FP32 contexts: GB300's FP64 rate is far
// lower), the eight warp results are combined in double by warp 0, then one
// atomic per block.  Must be called by every thread of the block.
template <typename T>
__device__ __forceinline__ double block_reduce_t(T v, bool is_max) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) {
        const T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? (u > v ? u : v) : v + u;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, r, o);
            r = is_max ? fmax(r, u) : r + u;
        }
    }
    return r;   // valid in thread 0
}

// ------------------------------------------------------------- fields
// mode 0: exchange only; mode 1: Hd + exchange + anisotropy + Zeeman
template <typename T, int MODE>
__global__ void k_field(Params<T> p, const T* __restrict__ m, const T* __restrict__ Hd, T* __restrict__ H) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    decompose(i, p.nx, p.ny, x, y, z);
    T Msi = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
    V3<T> h = {0, 0, 0};
    if (Msi != (T)0) {
        V3<T> mi = load3(m, i, p.N);
        h = exchange_at(p, m, i, x, y, z, mi, Msi);
        if (MODE == 1) {
            V3<T> l = local_at(p, mi, Msi);
            V3<T> d = load3(Hd, i, p.N);
            h = {h.x + l.x + d.x, h.y + l.y + d.y, h.z + l.z + d.z};
            if (p.dmi) {
                const V3<T> q = dmi_at(p, m, i, x, y, z, Msi);
                h = {h.x + q.x, h.y + q.y, h.z + q.z};
            }
        }
    } else if (MODE == 1) {
        h = load3(Hd, i, p.N);   // vacuum cell: only the stray (demag) field
    }
    store3(H, i, p.N, h);
}

// ------------------------------------------------------------- K7 stage
template <typename T, int METHOD, int S>
__global__ void k_stage(Params<T> p, const T* __restrict__ m_in, const T* __restrict__ Hd, const T* m0,
                        T* const* __restrict__ kbuf, T* m_out, Control* ctl) {
    constexpr int NS = rk_stages(METHOD);
    constexpr bool LAST = (S == NS - 1);
    if (ctl->status != 0 || ctl->done) return;
    const T dt = (T)ctl->dt;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double err = 0.0;
    if (i < p.N) {
        int x, y, z;
        decompose(i, p.nx, p.ny, x, y, z);
        T Msi = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
        V3<T> ks = {0, 0, 0};
        V3<T> mi = load3(m_in, i, p.N);
        if (Msi != (T)0) {
            V3<T> h = exchange_at(p, m_in, i, x, y, z, mi, Msi);
            V3<T> l = local_at(p, mi, Msi);
            V3<T> d = load3(Hd, i, p.N);
            h = {h.x + l.x + d.x, h.y + l.y + d.y, h.z + l.z + d.z};
            if (p.dmi) {
                const V3<T> q = dmi_at(p, m_in, i, x, y, z, Msi);
                h = {h.x + q.x, h.y + q.y, h.z + q.z};
            }
            ks = llg_rhs(p, mi, h);
            if (p.stt) {
                const V3<T> q = stt_at(p, mi, Msi);
                ks = {ks.x + q.x, ks.y + q.y, ks.z + q.z};
            }
        }
        V3<T> a0 = S == 0 ? mi : load3(m0, i, p.N);
        if constexpr (!LAST) {
            // next trial state m0 + dt sum_j a[S+1][j] k_j
            V3<T> acc = {0, 0, 0};
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const T c = (T)rk_a(METHOD, S + 1, j);
                if (c != (T)0) {
                    V3<T> kj = load3(kbuf[j], i, p.N);
                    acc.x += c * kj.x;
                    acc.y += c * kj.y;
                    acc.z += c * kj.z;
                }
            }
            const T cs = (T)rk_a(METHOD, S + 1, S);
            acc.x += cs * ks.x;
            acc.y += cs * ks.y;
            acc.z += cs * ks.z;
            store3(kbuf[S], i, p.N, ks);
            store3(m_out, i, p.N, V3<T>{a0.x + dt * acc.x, a0.y + dt * acc.y, a0.z + dt * acc.z});
        } else {
            V3<T> acc = {0, 0, 0}, e = {0, 0, 0};
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                const T cb = (T)rk_b(METHOD, j), ce = (T)rk_e(METHOD, j);
                if (cb != (T)0 || ce != (T)0) {
                    V3<T> kj = j == S ? ks : load3(kbuf[j], i, p.N);
                    acc.x += cb * kj.x;
                    acc.y += cb * kj.y;
                    acc.z += cb * kj.z;
                    e.x += ce * kj.x;
                    e.y += ce * kj.y;
                    e.z += ce * kj.z;
                }
            }
            V3<T> mn = {a0.x + dt * acc.x, a0.y + dt * acc.y, a0.z + dt * acc.z};
            T nrm = sqrt(mn.x * mn.x + mn.y * mn.y + mn.z * mn.z);
            if (Msi != (T)0 && nrm > (T)0) {
                T inv = (T)1 / nrm;
                mn = {mn.x * inv, mn.y * inv, mn.z * inv};
            }
            const bool bad = !(isfinite((double)mn.x) && isfinite((double)mn.y) && isfinite((double)mn.z));
            if (METHOD == MM_RKF45) {
                // a trial that overflowed is rejected (infinite error), as any too-large step
                err = (double)dt * (double)sqrt(e.x * e.x + e.y * e.y + e.z * e.z);
                if (bad || !isfinite(err)) err = INFINITY;
            } else if (bad) {
                atomicCAS(&ctl->status, 0, (int)MM_ERR_NONFINITE);
            }
            store3(m_out, i, p.N, mn);
        }
    }
    if constexpr (LAST && METHOD == MM_RKF45) block_max_atomic(err, &ctl->err_bits);
}

// K7, FP32, uniform material, nx % 4 == 0: four x-consecutive cells per
// thread with 16-byte loads and stores (the same arithmetic per cell as
// k_stage; the exchange weights A c_axis / Ms folded once).  Slope pointers
// travel by value.
struct KPtrs {
    float* k[6];
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& at(float4& v, int j) { return (&v.x)[j]; }
__device__ __forceinline__ float at(const float4& v, int j) { return (&v.x)[j]; }

struct Cells4 {
    float4 x, y, z;
};

__device__ __forceinline__ Cells4 ld_cells(const float* a, long i, long N) {
    return {ld4(a + i), ld4(a + i + N), ld4(a + i + 2 * N)};
}
__device__ __forceinline__ void st_cells(float* a, long i, long N, const Cells4& c) {
    st4(a + i, c.x);
    st4(a + i + N, c.y);
    st4(a + i + 2 * N, c.z);
}
// acc += w (nb - c), component-wise over the four cells
__device__ __forceinline__ void add_diff(Cells4& acc, const Cells4& nb, const Cells4& c, float w) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        at(acc.x, j) += w * (at(nb.x, j) - at(c.x, j));
        at(acc.y, j) += w * (at(nb.y, j) - at(c.y, j));
        at(acc.z, j) += w * (at(nb.z, j) - at(c.z, j));
    }
}

template <int METHOD, int S>
__global__ void __launch_bounds__(256) k_stage4(Params<float> p, float wx, float wy, float wz,
                                                const float* __restrict__ m_in, const float* __restrict__ Hd,
                                                const float* m0, KPtrs kb, float* m_out, Control* ctl) {
    constexpr int NS = rk_stages(METHOD);
    constexpr bool LAST = (S == NS - 1);
    if (ctl->status != 0 || ctl->done) return;
    const float dt = (float)ctl->dt;
    const long i = 4 * ((long)blockIdx.x * blockDim.x + threadIdx.x);
    const long N = p.N;
    double err = 0.0;
    if (i < N) {
        int x, y, z;
        decompose(i, p.nx, p.ny, x, y, z);
        const Cells4 c = ld_cells(m_in, i, N);
        Cells4 h = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
        // x neighbours: inside the quad, plus one cell on each side
        Cells4 xl, xr;
        xl.x = make_float4(x > 0 ? m_in[i - 1] : c.x.x, c.x.x, c.x.y, c.x.z);
        xl.y = make_float4(x > 0 ? m_in[i - 1 + N] : c.y.x, c.y.x, c.y.y, c.y.z);
        xl.z = make_float4(x > 0 ? m_in[i - 1 + 2 * N] : c.z.x, c.z.x, c.z.y, c.z.z);
        const bool rx = x + 4 < p.nx;
        xr.x = make_float4(c.x.y, c.x.z, c.x.w, rx ? m_in[i + 4] : c.x.w);
        xr.y = make_float4(c.y.y, c.y.z, c.y.w, rx ? m_in[i + 4 + N] : c.y.w);
        xr.z = make_float4(c.z.y, c.z.z, c.z.w, rx ? m_in[i + 4 + 2 * N] : c.z.w);
        add_diff(h, xl, c, wx);   // a missing neighbour contributes nb - c = 0
        add_diff(h, xr, c, wx);
        const long sy = p.nx, sz = (long)p.nx * p.ny;
        if (y > 0) add_diff(h, ld_cells(m_in, i - sy, N), c, wy);
        if (y < p.ny - 1) add_diff(h, ld_cells(m_in, i + sy, N), c, wy);
        if (z > 0) add_diff(h, ld_cells(m_in, i - sz, N), c, wz);
        if (z < p.nz - 1) add_diff(h, ld_cells(m_in, i + sz, N), c, wz);
        const Cells4 d = ld_cells(Hd, i, N);
        const Cells4 a0 = S == 0 ? c : ld_cells(m0, i, N);
        Cells4 ks;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const V3<float> mi = {at(c.x, j), at(c.y, j), at(c.z, j)};
            const V3<float> l = local_at(p, mi, p.Ms);
            const V3<float> H = {at(h.x, j) + l.x + at(d.x, j), at(h.y, j) + l.y + at(d.y, j),
                                 at(h.z, j) + l.z + at(d.z, j)};
            const V3<float> r = llg_rhs(p, mi, H);
            at(ks.x, j) = r.x;
            at(ks.y, j) = r.y;
            at(ks.z, j) = r.z;
        }
        if constexpr (!LAST) {
            Cells4 acc;
            const float cs = (float)rk_a(METHOD, S + 1, S);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                at(acc.x, j) = cs * at(ks.x, j);
                at(acc.y, j) = cs * at(ks.y, j);
                at(acc.z, j) = cs * at(ks.z, j);
            }
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const float cq = (float)rk_a(METHOD, S + 1, q);
                if (cq != 0.f) {
                    const Cells4 kq = ld_cells(kb.k[q], i, N);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        at(acc.x, j) += cq * at(kq.x, j);
                        at(acc.y, j) += cq * at(kq.y, j);
                        at(acc.z, j) += cq * at(kq.z, j);
                    }
                }
            }
            st_cells(kb.k[S], i, N, ks);
            Cells4 mo;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                at(mo.x, j) = at(a0.x, j) + dt * at(acc.x, j);
                at(mo.y, j) = at(a0.y, j) + dt * at(acc.y, j);
                at(mo.z, j) = at(a0.z, j) + dt * at(acc.z, j);
            }
            st_cells(m_out, i, N, mo);
        } else {
            Cells4 acc = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
            Cells4 e = acc;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const float cb = (float)rk_b(METHOD, q), ce = (float)rk_e(METHOD, q);
                if (cb != 0.f || ce != 0.f) {
                    const Cells4 kq = q == S ? ks : ld_cells(kb.k[q], i, N);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        at(acc.x, j) += cb * at(kq.x, j);
                        at(acc.y, j) += cb * at(kq.y, j);
                        at(acc.z, j) += cb * at(kq.z, j);
                        at(e.x, j) += ce * at(kq.x, j);
                        at(e.y, j) += ce * at(kq.y, j);
                        at(e.z, j) += ce * at(kq.z, j);
                    }
                }
            }
            Cells4 mo;
            bool bad = false;
            float e2 = 0.f;   // max |m5 - m4|^2 / dt^2 of the quad, in the path's precision
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float mx = at(a0.x, j) + dt * at(acc.x, j);
                float my = at(a0.y, j) + dt * at(acc.y, j);
                float mz = at(a0.z, j) + dt * at(acc.z, j);
                const float nrm = sqrtf(mx * mx + my * my + mz * mz);
                if (nrm > 0.f) {
                    const float inv = 1.f / nrm;
                    mx *= inv;
                    my *= inv;
                    mz *= inv;
                }
                bad |= !(isfinite(mx) && isfinite(my) && isfinite(mz));
                at(mo.x, j) = mx;
                at(mo.y, j) = my;
                at(mo.z, j) = mz;
                if (METHOD == MM_RKF45) {
                    const float v = at(e.x, j) * at(e.x, j) + at(e.y, j) * at(e.y, j) + at(e.z, j) * at(e.z, j);
                    bad |= !(v <= 3.0e38f);   // fmaxf would drop a NaN
                    e2 = fmaxf(e2, v);
                }
            }
            if (METHOD == MM_RKF45) {
                // one square root per thread (FP64 arithmetic is slow on this part)
                err = (double)dt * (double)sqrtf(e2);
                if (bad || !isfinite(err)) err = INFINITY;
            } else if (bad) {
                atomicCAS(&ctl->status, 0, (int)MM_ERR_NONFINITE);
            }
            st_cells(m_out, i, N, mo);
        }
    }
    if constexpr (LAST && METHOD == MM_RKF45) block_max_atomic(err, &ctl->err_bits);
}

// K7 in float-float arithmetic (MM_FFT_FF on an FP64 context), uniform
// material, no DMI or STT: the same per-cell arithmetic as k_stage on
// (h + l) float pairs (mm_ff.cuh), so the FP64 step runs on the FP32 pipes.
// Every array stays float64 (each value converted on load and on store); the
// RKF45 error is reduced as the squared norm per block, with one square root
// per block; the renormalisation uses a float-float Newton inverse square
// root started from rsqrtf.
struct KPtrsD {
    double* k[6];
};
struct FFStageCoef {
    ff wx, wy, wz;     // A (2 / (mu0 d^2)) / Ms per axis
    ff anis;           // 2 Ku / (mu0 Ms)
    ff ux, uy, uz, hx, hy, hz;
    ff pref, alpha;    // -gamma / (1 + alpha^2), alpha
};

__device__ __forceinline__ V3<ff> ld3ff(const double* __restrict__ a, long i, long N) {
    return {d2ff(a[i]), d2ff(a[i + N]), d2ff(a[i + 2 * N])};
}
__device__ __forceinline__ void st3ff(double* __restrict__ a, long i, long N, const V3<ff>& v) {
    a[i] = ff2d(v.x);
    a[i + N] = ff2d(v.y);
    a[i + 2 * N] = ff2d(v.z);
}
__device__ __forceinline__ ff half_of(ff a) { return ff(0.5f * a.h, 0.5f * a.l); }   // exact

template <int METHOD, int S>
__global__ void __launch_bounds__(256)
    k_stage_ff(FFStageCoef c, int nx, int ny, int nz, long N, const double* __restrict__ m_in,
               const double* __restrict__ Hd, const double* m0, KPtrsD kb, double* m_out, Control* ctl) {
    constexpr int NS = rk_stages(METHOD);
    constexpr bool LAST = (S == NS - 1);
    if (ctl->status != 0 || ctl->done) return;
    const ff dt = d2ff(ctl->dt);
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double w2 = 0.0;   // squared error norm of this cell (RKF45 last stage)
    if (i < N) {
        int x, y, z;
        decompose(i, nx, ny, x, y, z);
        const V3<ff> mi = ld3ff(m_in, i, N);
        // exchange (Eq. 2): sum over present neighbours w_axis (m_nb - m_i)
        V3<ff> h = {ff(0), ff(0), ff(0)};
        auto nb = [&](long j, ff w) {
            h.x += w * (d2ff(m_in[j]) - mi.x);
            h.y += w * (d2ff(m_in[j + N]) - mi.y);
            h.z += w * (d2ff(m_in[j + 2 * N]) - mi.z);
        };
        const long sy = nx, sz = (long)nx * ny;
        if (x > 0) nb(i - 1, c.wx);
        if (x < nx - 1) nb(i + 1, c.wx);
        if (y > 0) nb(i - sy, c.wy);
        if (y < ny - 1) nb(i + sy, c.wy);
        if (z > 0) nb(i - sz, c.wz);
        if (z < nz - 1) nb(i + sz, c.wz);
        // anisotropy, Zeeman, demag
        const ff k = c.anis * (mi.x * c.ux + mi.y * c.uy + mi.z * c.uz);
        const V3<ff> d = ld3ff(Hd, i, N);
        h = {h.x + (k * c.ux + c.hx) + d.x, h.y + (k * c.uy + c.hy) + d.y, h.z + (k * c.uz + c.hz) + d.z};
        // LLG right-hand side (Eq. 1)
        const V3<ff> a = {mi.y * h.z - mi.z * h.y, mi.z * h.x - mi.x * h.z, mi.x * h.y - mi.y * h.x};
        const V3<ff> b = {mi.y * a.z - mi.z * a.y, mi.z * a.x - mi.x * a.z, mi.x * a.y - mi.y * a.x};
        const V3<ff> ks = {c.pref * (a.x + c.alpha * b.x), c.pref * (a.y + c.alpha * b.y),
                           c.pref * (a.z + c.alpha * b.z)};
        const V3<ff> a0 = S == 0 ? mi : ld3ff(m0, i, N);
        if constexpr (!LAST) {
            V3<ff> acc = {ff(0), ff(0), ff(0)};
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const double cj = rk_a(METHOD, S + 1, j);
                if (cj != 0.0) {
                    const ff cf = ff(cj);
                    const V3<ff> kj = ld3ff(kb.k[j], i, N);
                    acc = {acc.x + cf * kj.x, acc.y + cf * kj.y, acc.z + cf * kj.z};
                }
            }
            const ff cs = ff(rk_a(METHOD, S + 1, S));
            acc = {acc.x + cs * ks.x, acc.y + cs * ks.y, acc.z + cs * ks.z};
            st3ff(kb.k[S], i, N, ks);
            st3ff(m_out, i, N, V3<ff>{a0.x + dt * acc.x, a0.y + dt * acc.y, a0.z + dt * acc.z});
        } else {
            V3<ff> acc = {ff(0), ff(0), ff(0)}, e = {ff(0), ff(0), ff(0)};
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                const double cb = rk_b(METHOD, j), ce = rk_e(METHOD, j);
                if (cb != 0.0 || ce != 0.0) {
                    const V3<ff> kj = j == S ? ks : ld3ff(kb.k[j], i, N);
                    const ff fb = ff(cb), fe = ff(ce);
                    acc = {acc.x + fb * kj.x, acc.y + fb * kj.y, acc.z + fb * kj.z};
                    e = {e.x + fe * kj.x, e.y + fe * kj.y, e.z + fe * kj.z};
                }
            }
            V3<ff> mn = {a0.x + dt * acc.x, a0.y + dt * acc.y, a0.z + dt * acc.z};
            const ff n2 = mn.x * mn.x + mn.y * mn.y + mn.z * mn.z;
            if (n2.h > 0.f && isfinite(n2.h)) {
                // y = 1 / sqrt(n2): rsqrtf start, two Newton steps y <- y (3/2 - n2 y^2 / 2)
                ff yv = ff(rsqrtf(n2.h));
                yv = yv * (ff(1.5) - half_of(n2 * (yv * yv)));
                yv = yv * (ff(1.5) - half_of(n2 * (yv * yv)));
                mn = {mn.x * yv, mn.y * yv, mn.z * yv};
            }
            const bool bad = !(isfinite(mn.x.h) && isfinite(mn.y.h) && isfinite(mn.z.h));
            if (METHOD == MM_RKF45) {
                w2 = ff2d(e.x * e.x + e.y * e.y + e.z * e.z);
                if (bad || !isfinite(w2)) w2 = INFINITY;
            } else if (bad) {
                atomicCAS(&ctl->status, 0, (int)MM_ERR_NONFINITE);
            }
            // |m| - 1 is now a few float-float units (~1e-14); one first-order
            // correction m (3/2 - |m|^2 / 2) in float64 leaves O(1e-28)
            double ox = ff2d(mn.x), oy = ff2d(mn.y), oz = ff2d(mn.z);
            if (!bad) {
                const double f = 1.5 - 0.5 * (ox * ox + oy * oy + oz * oz);
                ox *= f;
                oy *= f;
                oz *= f;
            }
            m_out[i] = ox;
            m_out[i + N] = oy;
            m_out[i + 2 * N] = oz;
        }
    }
    if constexpr (LAST && METHOD == MM_RKF45) {
        // block max of the squared norms; err = dt sqrt(max) for the controller
        __shared__ double red[32];
        for (int o = 16; o > 0; o >>= 1) w2 = fmax(w2, __shfl_xor_sync(0xffffffffu, w2, o));
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) red[w] = w2;
        __syncthreads();
        if (w == 0) {
            const int nw = (blockDim.x + 31) >> 5;
            w2 = lane < nw ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) w2 = fmax(w2, __shfl_xor_sync(0xffffffffu, w2, o));
            if (lane == 0 && w2 > 0.0) {
                const double err = ctl->dt * sqrt(w2);
                atomicMax(&ctl->err_bits, (unsigned long long)__double_as_longlong(err));
            }
        }
    }
}

// RKF45 step control on the device.
__global__ void k_controller(Control* ctl, int method) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (ctl->status != 0 || ctl->done) {
        ctl->accepted = 0;
        return;
    }
    const double dt = ctl->dt;
    if (method == MM_RK4) {
        ctl->accepted = 1;
        ctl->t += dt;
        ctl->steps += 1;
        ctl->dt_next = dt;
        return;
    }
    const double err = __longlong_as_double((long long)ctl->err_bits);
    const double tol = ctl->tol;
    const int acc = err <= tol;
    double fac;
    if (err <= 0.0) fac = 5.0;
    else fac = fmin(5.0, fmax(0.2, 0.9 * pow(tol / err, 0.2)));
    double dtn = dt * fac;
    ctl->accepted = acc;
    ctl->err_bits = 0ull;
    ctl->dt_next = dtn;
    if (acc) {
        ctl->t += dt;
        ctl->steps += 1;
        ctl->last_err = err;
    } else {
        ctl->rejects += 1;
    }
    if (dtn < 1e-20) {
        ctl->status = MM_ERR_DT_UNDERFLOW;
        return;
    }
    double rem = ctl->t_max - ctl->t;
    if (rem <= 0.0) {
        ctl->done = 1;
    } else if (dtn > rem) {
        dtn = rem;
    }
    ctl->dt = dtn;
}

template <typename T>
__global__ void k_commit(long n3, const T* __restrict__ src, T* __restrict__ dst, const Control* ctl) {
    if (!ctl->accepted) return;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) dst[i] = src[i];
}

// ------------------------------------------------------------- K9
template <typename T>
__global__ void k_energy(Params<T> p, const T* __restrict__ m, const T* __restrict__ Hd, double V, double mu0,
                         double Ku, Control* ctl) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double ed = 0, ex = 0, ea = 0, ez = 0, em = 0;
    if (i < p.N) {
        int x, y, z;
        decompose(i, p.nx, p.ny, x, y, z);
        T Msi = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
        if (Msi != (T)0) {
            V3<T> mi = load3(m, i, p.N);
            V3<T> h = exchange_at(p, m, i, x, y, z, mi, Msi);
            V3<T> d = load3(Hd, i, p.N);
            double ms = (double)Msi;
            ed = -0.5 * mu0 * V * ms * ((double)mi.x * d.x + (double)mi.y * d.y + (double)mi.z * d.z);
            ex = -0.5 * mu0 * V * ms * ((double)mi.x * h.x + (double)mi.y * h.y + (double)mi.z * h.z);
            double mu = (double)mi.x * p.ux + (double)mi.y * p.uy + (double)mi.z * p.uz;
            ea = -Ku * V * mu * mu;
            ez = -mu0 * V * ms * ((double)mi.x * p.hx + (double)mi.y * p.hy + (double)mi.z * p.hz);
            if (p.dmi) {
                const V3<T> q = dmi_at(p, m, i, x, y, z, Msi);
                em = -0.5 * mu0 * V * ms * ((double)mi.x * q.x + (double)mi.y * q.y + (double)mi.z * q.z);
            }
        }
    }
    block_sum_atomic(ed, &ctl->energy[0]);
    __syncthreads();
    block_sum_atomic(ex, &ctl->energy[1]);
    __syncthreads();
    block_sum_atomic(ea, &ctl->energy[2]);
    __syncthreads();
    block_sum_atomic(ez, &ctl->energy[3]);
    __syncthreads();
    block_sum_atomic(em, &ctl->energy[4]);
}

template <typename T>
__global__ void k_torque(Params<T> p, const T* __restrict__ m, const T* __restrict__ Hd, Control* ctl) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double tq = 0.0;
    if (i < p.N) {
        int x, y, z;
        decompose(i, p.nx, p.ny, x, y, z);
        T Msi = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
        if (Msi != (T)0) {
            V3<T> mi = load3(m, i, p.N);
            V3<T> h = exchange_at(p, m, i, x, y, z, mi, Msi);
            V3<T> l = local_at(p, mi, Msi);
            V3<T> d = load3(Hd, i, p.N);
            V3<T> q = {0, 0, 0};
            if (p.dmi) q = dmi_at(p, m, i, x, y, z, Msi);
            double Hx = (double)h.x + l.x + d.x + q.x, Hy = (double)h.y + l.y + d.y + q.y,
                   Hz = (double)h.z + l.z + d.z + q.z;
            double cx = mi.y * Hz - mi.z * Hy, cy = mi.z * Hx - mi.x * Hz, cz = mi.x * Hy - mi.y * Hx;
            tq = sqrt(cx * cx + cy * cy + cz * cz) / (double)Msi;
            if (!isfinite(tq)) tq = 1e300;
        }
    }
    block_max_atomic(tq, &ctl->torque_bits);
}

template <typename T>
__global__ void k_finite(long n3, const T* __restrict__ m, Control* ctl) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3 && !isfinite((double)m[i])) atomicCAS(&ctl->status, 0, (int)MM_ERR_NONFINITE);
}

constexpr int kThreads = 256;
inline unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// ------------------------------------------------ Barzilai-Borwein minimiser
// Steepest descent on the unit sphere with Barzilai-Borwein step lengths
// (the paper's minimiser, named beside RKF45 in its Implementation section):
// g = m x (m x h), h = H_eff / Ms; m <- normalise(m - tau g).  tau: 1e-4 on
// the first step, then (s.s)/(s.y) on odd and (s.y)/(y.y) on even steps
// (s = m_k - m_(k-1), y = g_k - g_(k-1), sums over all cells), or 1 where
// the quotient is not positive.  The step length and the stop test
// (max |m x H_eff| / Ms <= tol before a step) are taken on the device.
constexpr double kBBTau0 = 1e-4, kBBTauMax = 1.0;

template <typename T>
__global__ void k_bb_grad(Params<T> p, const T* __restrict__ m, const T* __restrict__ Hd, T* __restrict__ g,
                          const T* __restrict__ g_prev, const T* __restrict__ m_prev, int have_prev, Control* ctl) {
    if (ctl->status != 0 || ctl->done) return;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    T tq2 = 0, ss = 0, sy = 0, yy = 0;   // squared torque and the BB sums, in the path's type
    if (i < p.N) {
        int x, y, z;
        decompose(i, p.nx, p.ny, x, y, z);
        const T Msi = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
        V3<T> gi = {0, 0, 0};
        const V3<T> mi = load3(m, i, p.N);
        if (Msi != (T)0) {
            const V3<T> hx = exchange_at(p, m, i, x, y, z, mi, Msi);
            const V3<T> l = local_at(p, mi, Msi);
            const V3<T> d = load3(Hd, i, p.N);
            V3<T> q = {0, 0, 0};
            if (p.dmi) q = dmi_at(p, m, i, x, y, z, Msi);
            const T inv = (T)1 / Msi;
            const V3<T> h = {(hx.x + l.x + d.x + q.x) * inv, (hx.y + l.y + d.y + q.y) * inv,
                             (hx.z + l.z + d.z + q.z) * inv};
            const V3<T> a = {mi.y * h.z - mi.z * h.y, mi.z * h.x - mi.x * h.z, mi.x * h.y - mi.y * h.x};   // m x h
            gi = {mi.y * a.z - mi.z * a.y, mi.z * a.x - mi.x * a.z, mi.x * a.y - mi.y * a.x};            // m x (m x h)
            tq2 = a.x * a.x + a.y * a.y + a.z * a.z;
            if (!isfinite(tq2)) tq2 = sizeof(T) == 4 ? (T)3.0e38f : (T)1e300;
        }
        if (have_prev) {
            const V3<T> mp = load3(m_prev, i, p.N), gp = load3(g_prev, i, p.N);
            const T sx = mi.x - mp.x, sy_ = mi.y - mp.y, sz = mi.z - mp.z;
            const T yx = gi.x - gp.x, yy_ = gi.y - gp.y, yz = gi.z - gp.z;
            ss = sx * sx + sy_ * sy_ + sz * sz;
            sy = sx * yx + sy_ * yy_ + sz * yz;
            yy = yx * yx + yy_ * yy_ + yz * yz;
        }
        store3(g, i, p.N, gi);
    }
    // the torque maximum as the maximum squared norm, one square root per block
    const double t2 = block_reduce_t<T>(tq2, true);
    if (threadIdx.x == 0 && t2 > 0.0) {
        const double tq = t2 >= (sizeof(T) == 4 ? 3.0e38 : 1e300) ? 1e300 : sqrt(t2);
        atomicMax(&ctl->torque_bits, (unsigned long long)__double_as_longlong(tq));
    }
    if (have_prev) {
        const double a0 = block_reduce_t<T>(ss, false);
        if (threadIdx.x == 0) atomicAdd(&ctl->bb[0], a0);
        // s.y is a difference-like sum (the BB quotients divide by it and
        // read its sign), so its warp stage runs in double even in FP32
        const double a1 = block_reduce_t<double>((double)sy, false);
        if (threadIdx.x == 0) atomicAdd(&ctl->bb[1], a1);
        const double a2 = block_reduce_t<T>(yy, false);
        if (threadIdx.x == 0) atomicAdd(&ctl->bb[2], a2);
    }
}

// stop test and step length; ctl->dt carries tau to the update
__global__ void k_bb_tau(Control* ctl, double torque_tol, long max_iter) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || ctl->status != 0 || ctl->done) return;
    const double tq = __longlong_as_double((long long)ctl->torque_bits);
    const long k = (long)ctl->steps;
    if (tq <= torque_tol || k >= max_iter) {
        ctl->done = 1;
        return;
    }
    double tau = kBBTau0;
    if (k > 0) {
        const double q = (k & 1) ? ctl->bb[0] / ctl->bb[1] : ctl->bb[1] / ctl->bb[2];
        tau = (isfinite(q) && q > 0.0) ? q : kBBTauMax;
    }
    ctl->dt = tau;
    ctl->steps = k + 1;
    ctl->torque_bits = 0ull;
    ctl->bb[0] = ctl->bb[1] = ctl->bb[2] = 0.0;
}

template <typename T>
__global__ void k_bb_update(Params<T> p, T* __restrict__ m, const T* __restrict__ g, T* __restrict__ m_prev,
                            const Control* ctl) {
    if (ctl->status != 0 || ctl->done) return;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const T tau = (T)ctl->dt;
    const V3<T> mi = load3(m, i, p.N);
    store3(m_prev, i, p.N, mi);
    const T Msi = p.Ms_cell ? p.Ms_cell[i] : p.Ms;
    if (Msi == (T)0) return;   // vacuum cells do not move
    const V3<T> gi = load3(g, i, p.N);
    V3<T> mn = {mi.x - tau * gi.x, mi.y - tau * gi.y, mi.z - tau * gi.z};
    const T nrm = sqrt(mn.x * mn.x + mn.y * mn.y + mn.z * mn.z);
    if (nrm > (T)0) mn = {mn.x / nrm, mn.y / nrm, mn.z / nrm};
    store3(m, i, p.N, mn);
}

template <typename T, int METHOD, int S>
int launch_stage(mm_ctx* ctx, const Params<T>& p, const void* m_in, const void* m0, void* m_out, T* const* kdev) {
    KernelTimer kt(ctx, MM_K_STAGE);
    if constexpr (sizeof(T) == 8) {
        if (ctx->fft_mode == MM_FFT_FF && !p.Ms_cell && !p.A_cell && p.Ms != 0.0 && !p.dmi && !p.stt) {
            KPtrsD kb;
            for (int s = 0; s < 6; ++s) kb.k[s] = (double*)ctx->k[s];
            const double inv = 1.0 / (double)p.Ms;
            FFStageCoef c;
            c.wx = ff((double)(p.A * p.cx) * inv);
            c.wy = ff((double)(p.A * p.cy) * inv);
            c.wz = ff((double)(p.A * p.cz) * inv);
            c.anis = ff((double)p.anis * inv);
            c.ux = ff((double)p.ux);
            c.uy = ff((double)p.uy);
            c.uz = ff((double)p.uz);
            c.hx = ff((double)p.hx);
            c.hy = ff((double)p.hy);
            c.hz = ff((double)p.hz);
            c.pref = ff((double)p.pref);
            c.alpha = ff((double)p.alpha);
            k_stage_ff<METHOD, S><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(
                c, p.nx, p.ny, p.nz, p.N, (const double*)m_in, (const double*)ctx->Hd, (const double*)m0, kb,
                (double*)m_out, ctx->ctl);
            MM_LAUNCH_CHECK(ctx);
            return MM_OK;
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (!p.Ms_cell && !p.A_cell && p.Ms != 0.f && p.nx % 4 == 0 && !p.dmi && !p.stt) {
            KPtrs kb;
            for (int s = 0; s < 6; ++s) kb.k[s] = (float*)ctx->k[s];
            const float inv = 1.f / p.Ms;
            k_stage4<METHOD, S><<<blocks_for(p.N / 4), kThreads, 0, ctx->stream>>>(
                p, p.A * p.cx * inv, p.A * p.cy * inv, p.A * p.cz * inv, (const float*)m_in, (const float*)ctx->Hd,
                (const float*)m0, kb, (float*)m_out, ctx->ctl);
            MM_LAUNCH_CHECK(ctx);
            return MM_OK;
        }
    }
    k_stage<T, METHOD, S><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (const T*)m_in, (const T*)ctx->Hd,
                                                                          (const T*)m0, kdev, (T*)m_out, ctx->ctl);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <typename T, int METHOD>
int stage_dispatch(mm_ctx* ctx, int s, const void* m_in, const void* m0, void* m_out) {
    Params<T> p = make_params<T>(ctx);
    T* const* kdev = (T* const*)ctx->kptrs;
    switch (s) {
        case 0: return launch_stage<T, METHOD, 0>(ctx, p, m_in, m0, m_out, kdev);
        case 1: return launch_stage<T, METHOD, 1>(ctx, p, m_in, m0, m_out, kdev);
        case 2: return launch_stage<T, METHOD, 2>(ctx, p, m_in, m0, m_out, kdev);
        case 3: return launch_stage<T, METHOD, 3>(ctx, p, m_in, m0, m_out, kdev);
        case 4:
            if constexpr (METHOD == MM_RKF45) return launch_stage<T, METHOD, 4>(ctx, p, m_in, m0, m_out, kdev);
            break;
        case 5:
            if constexpr (METHOD == MM_RKF45) return launch_stage<T, METHOD, 5>(ctx, p, m_in, m0, m_out, kdev);
            break;
    }
    return fail(ctx, MM_ERR_INVALID_ARG, "bad stage %d", s);
}

template <typename T>
int exchange_t(mm_ctx* ctx, const void* m, void* H) {
    KernelTimer kt(ctx, MM_K_REDUCE);
    Params<T> p = make_params<T>(ctx);
    k_field<T, 0><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (const T*)m, nullptr, (T*)H);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}
template <typename T>
int effective_t(mm_ctx* ctx, const void* m, const void* Hd, void* H) {
    KernelTimer kt(ctx, MM_K_REDUCE);
    Params<T> p = make_params<T>(ctx);
    k_field<T, 1><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (const T*)m, (const T*)Hd, (T*)H);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}
template <typename T>
int energy_t(mm_ctx* ctx, const void* m, const void* Hd) {
    KernelTimer kt(ctx, MM_K_REDUCE);
    Params<T> p = make_params<T>(ctx);
    double V = ctx->dx * ctx->dy * ctx->dz;
    k_energy<T><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (const T*)m, (const T*)Hd, V, kMu0, ctx->Ku, ctx->ctl);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}
template <typename T>
int torque_t(mm_ctx* ctx, const void* m, const void* Hd) {
    KernelTimer kt(ctx, MM_K_REDUCE);
    Params<T> p = make_params<T>(ctx);
    k_torque<T><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (const T*)m, (const T*)Hd, ctx->ctl);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace

int field_exchange(mm_ctx* ctx, const void* m, void* H) {
    return ctx->prec == MM_F64 ? exchange_t<double>(ctx, m, H) : exchange_t<float>(ctx, m, H);
}
int field_effective(mm_ctx* ctx, const void* m, const void* Hd, void* H) {
    return ctx->prec == MM_F64 ? effective_t<double>(ctx, m, Hd, H) : effective_t<float>(ctx, m, Hd, H);
}

int energy_launch(mm_ctx* ctx, const void* m, const void* Hd) {
    return ctx->prec == MM_F64 ? energy_t<double>(ctx, m, Hd) : energy_t<float>(ctx, m, Hd);
}
int torque_launch(mm_ctx* ctx, const void* m, const void* Hd) {
    return ctx->prec == MM_F64 ? torque_t<double>(ctx, m, Hd) : torque_t<float>(ctx, m, Hd);
}

int rk_stage(mm_ctx* ctx, int method, int s, const void* m_in, const void* m0, void* m_out) {
    if (ctx->prec == MM_F64) {
        return method == MM_RK4 ? stage_dispatch<double, MM_RK4>(ctx, s, m_in, m0, m_out)
                                : stage_dispatch<double, MM_RKF45>(ctx, s, m_in, m0, m_out);
    }
    return method == MM_RK4 ? stage_dispatch<float, MM_RK4>(ctx, s, m_in, m0, m_out)
                            : stage_dispatch<float, MM_RKF45>(ctx, s, m_in, m0, m_out);
}

int rk_controller(mm_ctx* ctx, int method) {
    KernelTimer kt(ctx, MM_K_CONTROL);
    k_controller<<<1, 32, 0, ctx->stream>>>(ctx->ctl, method);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int rk_commit(mm_ctx* ctx, void* m0) {
    KernelTimer kt(ctx, MM_K_CONTROL);
    long n3 = 3 * ctx->N;
    if (ctx->prec == MM_F64)
        k_commit<double><<<blocks_for(n3), kThreads, 0, ctx->stream>>>(n3, (const double*)ctx->mnext, (double*)m0, ctx->ctl);
    else
        k_commit<float><<<blocks_for(n3), kThreads, 0, ctx->stream>>>(n3, (const float*)ctx->mnext, (float*)m0, ctx->ctl);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <typename T>
int bb_iteration_t(mm_ctx* ctx, void* m, void* g, const void* g_prev, void* m_prev, bool have_prev, double tol,
                   long max_iter) {
    KernelTimer kt(ctx, MM_K_REDUCE);
    const Params<T> p = make_params<T>(ctx);
    k_bb_grad<T><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (const T*)m, (const T*)ctx->Hd, (T*)g,
                                                                (const T*)g_prev, (const T*)m_prev, have_prev ? 1 : 0,
                                                                ctx->ctl);
    k_bb_tau<<<1, 32, 0, ctx->stream>>>(ctx->ctl, tol, max_iter);
    k_bb_update<T><<<blocks_for(p.N), kThreads, 0, ctx->stream>>>(p, (T*)m, (const T*)g, (T*)m_prev, ctx->ctl);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

int bb_iteration(mm_ctx* ctx, void* m, void* g, const void* g_prev, void* m_prev, bool have_prev, double torque_tol,
                 long max_iter) {
    return ctx->prec == MM_F64 ? bb_iteration_t<double>(ctx, m, g, g_prev, m_prev, have_prev, torque_tol, max_iter)
                               : bb_iteration_t<float>(ctx, m, g, g_prev, m_prev, have_prev, torque_tol, max_iter);
}

int check_finite_launch(mm_ctx* ctx, const void* m) {
    KernelTimer kt(ctx, MM_K_REDUCE);
    long n3 = 3 * ctx->N;
    if (ctx->prec == MM_F64)
        k_finite<double><<<blocks_for(n3), kThreads, 0, ctx->stream>>>(n3, (const double*)m, ctx->ctl);
    else
        k_finite<float><<<blocks_for(n3), kThreads, 0, ctx->stream>>>(n3, (const float*)m, ctx->ctl);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace mm
