// Hand-written adjoints: vector-Jacobian products of the demag field, the
// exchange field and one RK4 step of the LLG equation with respect to the
// magnetisation and the per-cell saturation magnetisation Ms.
//
// With f(m; Ms) = pref [m x H + alpha m x (m x H)], pref = -gamma/(1+alpha^2)
// (Eq. 1 for unit m) and H = H_d + H_ex + H_anis + H_ext, the product of a
// cotangent w with the Jacobian is, per cell,
//   g_H = pref [w x m + alpha (w x m) x m]                    (through H)
//   g_m = pref [H x w + alpha ((m x H) x w + H x (w x m))]    (m explicit)
// and g_H is pulled back through each field term:
//   demag  H_d = -N * (Ms m): N is symmetric and even, so the operator is
//          self-adjoint and d<g,H_d>/dm = Ms (-N * g), d/dMs = m . (-N * g)
//          (one demag convolution of g with Ms = 1);
//   exchange H_ex = E(m) / Ms with E the symmetric 6-point stencil
//          (harmonic-mean A, vacuum bonds removed): d/dm = E(g / Ms),
//          d/dMs = -g . H_ex / Ms;
//   anisotropy H_an = 2 Ku/(mu0 Ms) (m.u) u: d/dm = 2 Ku/(mu0 Ms) (g.u) u,
//          d/dMs = -g . H_an / Ms.
// The RK4 step (classic tableau, then m <- u / |u|) is reversed stage by
// stage from its stage states (recorded while the checkpoint segment is
// replayed, or recomputed from m_n); the renormalisation pulls back as
// (lam - (lam . m_out) m_out) / |u|.
#include <algorithm>
#include <cmath>

#include "mm_fields.cuh"

namespace mm {
namespace {

constexpr int kT = 256;
// largest forward tape a trajectory VJP allocates (bytes)
constexpr size_t kTapeBudget = (size_t)16 << 30;
inline unsigned nblk(long n) { return (unsigned)((n + kT - 1) / kT); }

template <typename T> __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T> __device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> __device__ __forceinline__ V3<T> axpy(T a, V3<T> x, V3<T> y) {
    return {a * x.x + y.x, a * x.y + y.y, a * x.z + y.z};
}
template <typename T> __device__ __forceinline__ T ms_at(const Params<T>& p, long i) {
    return p.Ms_cell ? p.Ms_cell[i] : p.Ms;
}

// E(q)_i = sum over magnetic neighbours of c A_h (q_nb - q_i), q = g / Ms
template <typename T>
__device__ __forceinline__ V3<T> stencil_g_over_ms(const Params<T>& p, const T* __restrict__ g, long i, int x, int y,
                                                   int z, T Msi) {
    const T Ai = p.A_cell ? p.A_cell[i] : p.A;
    const T inv_i = (T)1 / Msi;
    const V3<T> qi = {g[i] * inv_i, g[i + p.N] * inv_i, g[i + 2 * p.N] * inv_i};
    V3<T> acc = {0, 0, 0};
    auto nb = [&](long j, T c) {
        T Msj = ms_at(p, j);
        if (Msj == (T)0) return;
        T Ah;
        if (p.A_cell) {
            T Aj = p.A_cell[j];
            T s = Ai + Aj;
            Ah = s > (T)0 ? (T)2 * Ai * Aj / s : (T)0;
        } else {
            Ah = p.A;
        }
        const T w = Ah * c, inv_j = (T)1 / Msj;
        acc.x += w * (g[j] * inv_j - qi.x);
        acc.y += w * (g[j + p.N] * inv_j - qi.y);
        acc.z += w * (g[j + 2 * p.N] * inv_j - qi.z);
    };
    const long sy = p.nx, sz = (long)p.nx * p.ny;
    if (x > 0) nb(i - 1, p.cx);
    if (x < p.nx - 1) nb(i + 1, p.cx);
    if (y > 0) nb(i - sy, p.cy);
    if (y < p.ny - 1) nb(i + sy, p.cy);
    if (z > 0) nb(i - sz, p.cz);
    if (z < p.nz - 1) nb(i + sz, p.cz);
    return acc;
}

// u = m0 + dt sum_s b_s k_s with k_3 = f(X_3) formed here; lam <- pull-back
// of the renormalisation; lk[s] <- b_s dt lam_u.
template <typename T>
__global__ void k_vjp_norm(Params<T> p, const T* __restrict__ m0, const T* __restrict__ k0, const T* __restrict__ k1,
                           const T* __restrict__ k2, const T* __restrict__ x3, const T* __restrict__ hd3, T dt,
                           T* __restrict__ lam, T* __restrict__ lk0, T* __restrict__ lk1, T* __restrict__ lk2,
                           T* __restrict__ lk3) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    decompose(i, p.nx, p.ny, x, y, z);
    const T Msi = ms_at(p, i);
    V3<T> lu = {0, 0, 0};
    if (Msi != (T)0) {
        V3<T> X3 = load3(x3, i, p.N);
        V3<T> h = exchange_at(p, x3, i, x, y, z, X3, Msi);
        V3<T> l = local_at(p, X3, Msi);
        V3<T> d = load3(hd3, i, p.N);
        V3<T> k3 = llg_rhs(p, X3, V3<T>{h.x + l.x + d.x, h.y + l.y + d.y, h.z + l.z + d.z});
        V3<T> a = load3(k0, i, p.N), b = load3(k1, i, p.N), c = load3(k2, i, p.N), m = load3(m0, i, p.N);
        const T s6 = dt / (T)6, s3 = dt / (T)3;
        V3<T> u = {m.x + s6 * (a.x + k3.x) + s3 * (b.x + c.x), m.y + s6 * (a.y + k3.y) + s3 * (b.y + c.y),
                   m.z + s6 * (a.z + k3.z) + s3 * (b.z + c.z)};
        const T nu = sqrt(dot(u, u));
        const V3<T> mo = {u.x / nu, u.y / nu, u.z / nu};
        const V3<T> L = load3(lam, i, p.N);
        const T lm = dot(L, mo);
        lu = {(L.x - lm * mo.x) / nu, (L.y - lm * mo.y) / nu, (L.z - lm * mo.z) / nu};
    }
    store3(lam, i, p.N, lu);
    const T s6 = dt / (T)6, s3 = dt / (T)3;
    store3(lk0, i, p.N, V3<T>{s6 * lu.x, s6 * lu.y, s6 * lu.z});
    store3(lk1, i, p.N, V3<T>{s3 * lu.x, s3 * lu.y, s3 * lu.z});
    store3(lk2, i, p.N, V3<T>{s3 * lu.x, s3 * lu.y, s3 * lu.z});
    store3(lk3, i, p.N, V3<T>{s6 * lu.x, s6 * lu.y, s6 * lu.z});
}

// first half of the RHS pull-back at state X with cotangent w:
// G = g_H, P = g_m (explicit m dependence)
template <typename T>
__global__ void k_vjp_rhs_a(Params<T> p, const T* __restrict__ X, const T* __restrict__ hd, const T* __restrict__ w,
                            T* __restrict__ G, T* __restrict__ P) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    decompose(i, p.nx, p.ny, x, y, z);
    const T Msi = ms_at(p, i);
    V3<T> gH = {0, 0, 0}, gm = {0, 0, 0};
    if (Msi != (T)0) {
        V3<T> m = load3(X, i, p.N);
        V3<T> h = exchange_at(p, X, i, x, y, z, m, Msi);
        V3<T> l = local_at(p, m, Msi);
        V3<T> d = load3(hd, i, p.N);
        V3<T> H = {h.x + l.x + d.x, h.y + l.y + d.y, h.z + l.z + d.z};
        V3<T> W = load3(w, i, p.N);
        V3<T> wm = cross(W, m);
        V3<T> wmm = cross(wm, m);
        gH = {p.pref * (wm.x + p.alpha * wmm.x), p.pref * (wm.y + p.alpha * wmm.y), p.pref * (wm.z + p.alpha * wmm.z)};
        V3<T> a = cross(m, H);
        V3<T> t1 = cross(H, W), t2 = cross(a, W), t3 = cross(H, wm);
        gm = {p.pref * (t1.x + p.alpha * (t2.x + t3.x)), p.pref * (t1.y + p.alpha * (t2.y + t3.y)),
              p.pref * (t1.z + p.alpha * (t2.z + t3.z))};
    }
    store3(G, i, p.N, gH);
    store3(P, i, p.N, gm);
}

// second half: lam_X = P + Ms D + E(G/Ms) + anisotropy pull-back;
// lam += lam_X; lk_prev += coef lam_X (if lk_prev); gMs += m.D - G.(H_ex + H_an)/Ms
template <typename T>
__global__ void k_vjp_rhs_b(Params<T> p, const T* __restrict__ X, const T* __restrict__ G, const T* __restrict__ P,
                            const T* __restrict__ D, T* __restrict__ lam, T* __restrict__ lk_prev, T coef,
                            T* __restrict__ gMs) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    decompose(i, p.nx, p.ny, x, y, z);
    const T Msi = ms_at(p, i);
    if (Msi == (T)0) return;
    V3<T> m = load3(X, i, p.N);
    V3<T> g = load3(G, i, p.N);
    V3<T> dd = load3(D, i, p.N);
    V3<T> e = stencil_g_over_ms(p, G, i, x, y, z, Msi);
    const T ka = p.anis / Msi;
    const T gu = g.x * p.ux + g.y * p.uy + g.z * p.uz;
    V3<T> pr = load3(P, i, p.N);
    V3<T> lx = {pr.x + Msi * dd.x + e.x + ka * gu * p.ux, pr.y + Msi * dd.y + e.y + ka * gu * p.uy,
                pr.z + Msi * dd.z + e.z + ka * gu * p.uz};
    V3<T> L = load3(lam, i, p.N);
    store3(lam, i, p.N, V3<T>{L.x + lx.x, L.y + lx.y, L.z + lx.z});
    if (lk_prev) {
        V3<T> K = load3(lk_prev, i, p.N);
        store3(lk_prev, i, p.N, axpy(coef, lx, K));
    }
    // Ms pull-back: demag through M = Ms m, exchange and anisotropy through 1/Ms
    V3<T> hex = exchange_at(p, X, i, x, y, z, m, Msi);
    const T mu = m.x * p.ux + m.y * p.uy + m.z * p.uz;
    V3<T> han = {ka * mu * p.ux, ka * mu * p.uy, ka * mu * p.uz};
    gMs[i] += dot(m, dd) - (dot(g, hex) + dot(g, han)) / Msi;
}

// transposes of the single field terms (autograd of demag_field / exchange_field)
template <typename T>
__global__ void k_demag_vjp(Params<T> p, const T* __restrict__ m, const T* __restrict__ D, T* __restrict__ gm,
                            T* __restrict__ gMs) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const T Msi = ms_at(p, i);
    V3<T> dd = load3(D, i, p.N);
    store3(gm, i, p.N, V3<T>{Msi * dd.x, Msi * dd.y, Msi * dd.z});
    if (gMs) gMs[i] += dot(load3(m, i, p.N), dd);
}

template <typename T>
__global__ void k_exchange_vjp(Params<T> p, const T* __restrict__ m, const T* __restrict__ g, T* __restrict__ gm,
                               T* __restrict__ gMs) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    decompose(i, p.nx, p.ny, x, y, z);
    const T Msi = ms_at(p, i);
    if (Msi == (T)0) {
        store3(gm, i, p.N, V3<T>{0, 0, 0});
        return;
    }
    store3(gm, i, p.N, stencil_g_over_ms(p, g, i, x, y, z, Msi));
    if (gMs) {
        V3<T> mi = load3(m, i, p.N);
        gMs[i] += -dot(load3(g, i, p.N), exchange_at(p, m, i, x, y, z, mi, Msi)) / Msi;
    }
}

constexpr int kAdjFields = 14;

int ensure_workspace(mm_ctx* ctx) {
    if (ctx->adj) return MM_OK;
    const size_t e = ctx->prec == MM_F64 ? sizeof(double) : sizeof(float);
    const size_t bytes = (size_t)kAdjFields * 3 * ctx->N * e;
    cudaError_t ce = cudaMalloc(&ctx->adj, bytes);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        ctx->adj = nullptr;
        return fail(ctx, MM_ERR_NOMEM, "adjoint workspace (%zu bytes): %s", bytes, cudaGetErrorString(ce));
    }
    return MM_OK;
}

// One RK4 step's forward record, written while a checkpoint segment is
// replayed so the step VJP need not recompute it: the stage states X1..X3,
// the demag fields of X0..X3 and the slopes k0..k2.
struct StepTape {
    void* X[3];
    void* H[4];
    void* k[3];
};

// One RK4 step from m, recording its tape; m_next = NULL stops after the
// demag field of X3 (the last step of a segment, whose successor is known).
int rk4_step_record(mm_ctx* ctx, const void* m, void* m_next, const StepTape& tp) {
    const size_t v = 3 * (size_t)ctx->N * (ctx->prec == MM_F64 ? sizeof(double) : sizeof(float));
    void* hd_saved = ctx->Hd;
    int rc = MM_OK;
    const void* Xs = m;
    for (int s = 0; s < 4 && rc == MM_OK; ++s) {
        ctx->Hd = tp.H[s];
        rc = demag_apply(ctx, Xs, tp.H[s]);
        if (rc || (s == 3 && !m_next)) break;
        void* out = s < 3 ? tp.X[s] : m_next;
        rc = rk_stage(ctx, MM_RK4, s, Xs, m, out);
        if (!rc && s < 3) {
            cudaError_t ce = cudaMemcpyAsync(tp.k[s], ctx->k[s], v, cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce != cudaSuccess) rc = fail(ctx, MM_ERR_CUDA, "tape copy: %s", cudaGetErrorString(ce));
        }
        Xs = out;
    }
    ctx->Hd = hd_saved;
    return rc;
}

// reset: put dt into the control block first (a standalone call); the
// trajectory VJP sets it once for all its steps.  tape: the step's forward
// record, or NULL to recompute it here.
template <typename T>
int step_vjp(mm_ctx* ctx, const T* m0, double dt, T* lam, T* gMs, const StepTape* tape = nullptr, bool reset = true) {
    int rc = ensure_workspace(ctx);
    if (rc) return rc;
    const long n3 = 3 * ctx->N;
    T* w = (T*)ctx->adj;
    T* X[4] = {(T*)m0, w, w + n3, w + 2 * n3};            // stage states
    T* Hst[4] = {w + 3 * n3, w + 4 * n3, w + 5 * n3, w + 6 * n3};
    T* lk[4] = {w + 7 * n3, w + 8 * n3, w + 9 * n3, w + 10 * n3};
    T* G = w + 11 * n3;
    T* P = w + 12 * n3;
    T* D = w + 13 * n3;
    const T* kk[3] = {(const T*)ctx->k[0], (const T*)ctx->k[1], (const T*)ctx->k[2]};
    if (reset && (rc = ctl_reset_push(ctx, 0.0, dt, INFINITY, 1.0))) return rc;
    if (tape) {
        for (int s = 0; s < 3; ++s) {
            X[s + 1] = (T*)tape->X[s];
            kk[s] = (const T*)tape->k[s];
        }
        for (int s = 0; s < 4; ++s) Hst[s] = (T*)tape->H[s];
    } else {
        // recompute the stage states X_s and their demag fields
        void* hd_saved = ctx->Hd;
        for (int s = 0; s < 3 && rc == MM_OK; ++s) {
            ctx->Hd = Hst[s];
            rc = demag_apply(ctx, X[s], Hst[s]);
            if (!rc) rc = rk_stage(ctx, MM_RK4, s, X[s], m0, X[s + 1]);
        }
        ctx->Hd = hd_saved;
        if (rc) return rc;
        if ((rc = demag_apply(ctx, X[3], Hst[3]))) return rc;
    }
    Params<T> p = make_params<T>(ctx);
    {
        KernelTimer kt(ctx, MM_K_STAGE);
        k_vjp_norm<T><<<nblk(ctx->N), kT, 0, ctx->stream>>>(p, m0, kk[0], kk[1], kk[2], X[3], Hst[3], (T)dt, lam,
                                                            lk[0], lk[1], lk[2], lk[3]);
        MM_LAUNCH_CHECK(ctx);
    }
    // classic RK4: X_1 = m0 + dt/2 k_0, X_2 = m0 + dt/2 k_1, X_3 = m0 + dt k_2
    const double coef[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};
    for (int s = 3; s >= 0; --s) {
        {
            KernelTimer kt(ctx, MM_K_STAGE);
            k_vjp_rhs_a<T><<<nblk(ctx->N), kT, 0, ctx->stream>>>(p, X[s], Hst[s], lk[s], G, P);
            MM_LAUNCH_CHECK(ctx);
        }
        if ((rc = demag_apply_unit(ctx, G, D))) return rc;
        {
            KernelTimer kt(ctx, MM_K_STAGE);
            k_vjp_rhs_b<T><<<nblk(ctx->N), kT, 0, ctx->stream>>>(p, X[s], G, P, D, lam, s > 0 ? lk[s - 1] : nullptr,
                                                                 (T)coef[s], gMs);
            MM_LAUNCH_CHECK(ctx);
        }
    }
    return MM_OK;
}

template <typename T>
int demag_vjp_t(mm_ctx* ctx, const T* g, const T* m, T* gm, T* gMs) {
    int rc = ensure_workspace(ctx);
    if (rc) return rc;
    T* D = (T*)ctx->adj + 13 * 3 * ctx->N;
    if ((rc = demag_apply_unit(ctx, g, D))) return rc;
    Params<T> p = make_params<T>(ctx);
    KernelTimer kt(ctx, MM_K_REDUCE);
    k_demag_vjp<T><<<nblk(ctx->N), kT, 0, ctx->stream>>>(p, m, D, gm, gMs);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

template <typename T>
int exchange_vjp_t(mm_ctx* ctx, const T* g, const T* m, T* gm, T* gMs) {
    Params<T> p = make_params<T>(ctx);
    KernelTimer kt(ctx, MM_K_REDUCE);
    k_exchange_vjp<T><<<nblk(ctx->N), kT, 0, ctx->stream>>>(p, m, g, gm, gMs);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

// n fixed RK4 steps of m in place, no host synchronisation (the caller's
// control block must hold dt)
int rk4_steps(mm_ctx* ctx, void* m, long n) {
    int rc;
    for (long k = 0; k < n; ++k) {
        for (int s = 0; s < 4; ++s) {
            const void* m_in = s == 0 ? m : ctx->ms[s % 2];
            void* m_out = s < 3 ? ctx->ms[(s + 1) % 2] : m;
            if ((rc = demag_apply(ctx, m_in, ctx->Hd))) return rc;
            if ((rc = rk_stage(ctx, MM_RK4, s, m_in, m, m_out))) return rc;
        }
    }
    return MM_OK;
}

int status_check(mm_ctx* ctx) {
    int rc = ctl_pull(ctx);
    if (rc) return rc;
    if (ctx->ctl_host->status)
        return fail(ctx, ctx->ctl_host->status, "NaN or Inf in the magnetisation during RK4 steps");
    return MM_OK;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" {

int mm_rk4_step_vjp(mm_ctx* ctx, const void* m0, double dt, void* lam, void* gMs) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!m0 || !lam || !gMs) return fail(ctx, MM_ERR_INVALID_ARG, "m0, lam and gMs must be device pointers");
    if (!(std::isfinite(dt) && dt > 0)) return fail(ctx, MM_ERR_INVALID_ARG, "dt must be > 0");
    if (ctx->D != 0.0 || ctx->stt_on) return fail(ctx, MM_ERR_INVALID_ARG, "the adjoint covers neither DMI nor STT");
    MM_BIND(ctx);
    if (ctx->prec == MM_F64) return step_vjp<double>(ctx, (const double*)m0, dt, (double*)lam, (double*)gMs);
    return step_vjp<float>(ctx, (const float*)m0, dt, (float*)lam, (float*)gMs);
}

int mm_demag_vjp(mm_ctx* ctx, const void* g, const void* m, void* gm, void* gMs) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!g || !m || !gm) return fail(ctx, MM_ERR_INVALID_ARG, "g, m and gm must be device pointers");
    MM_BIND(ctx);
    if (ctx->prec == MM_F64)
        return demag_vjp_t<double>(ctx, (const double*)g, (const double*)m, (double*)gm, (double*)gMs);
    return demag_vjp_t<float>(ctx, (const float*)g, (const float*)m, (float*)gm, (float*)gMs);
}

int mm_exchange_vjp(mm_ctx* ctx, const void* g, const void* m, void* gm, void* gMs) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!g || !m || !gm) return fail(ctx, MM_ERR_INVALID_ARG, "g, m and gm must be device pointers");
    MM_BIND(ctx);
    if (ctx->prec == MM_F64)
        return exchange_vjp_t<double>(ctx, (const double*)g, (const double*)m, (double*)gm, (double*)gMs);
    return exchange_vjp_t<float>(ctx, (const float*)g, (const float*)m, (float*)gm, (float*)gMs);
}

int mm_rk4_trajectory(mm_ctx* ctx, void* m, double dt, long nsteps) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!m || nsteps < 0 || !(std::isfinite(dt) && dt > 0))
        return fail(ctx, MM_ERR_INVALID_ARG, "m must be a device pointer, dt > 0, nsteps >= 0");
    MM_BIND(ctx);
    int rc = ctl_reset_push(ctx, 0.0, dt, INFINITY, 1.0);
    if (!rc) rc = check_finite_launch(ctx, m);
    if (!rc) rc = rk4_steps(ctx, m, nsteps);
    if (!rc) rc = status_check(ctx);
    return rc;
}

int mm_rk4_trajectory_vjp(mm_ctx* ctx, const void* m0, double dt, long nsteps, void* lam, void* gMs,
                          long checkpoint_every) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!m0 || !lam || !gMs || nsteps < 0 || !(std::isfinite(dt) && dt > 0))
        return fail(ctx, MM_ERR_INVALID_ARG, "device pointers, dt > 0 and nsteps >= 0 required");
    if (ctx->D != 0.0 || ctx->stt_on) return fail(ctx, MM_ERR_INVALID_ARG, "the adjoint covers neither DMI nor STT");
    MM_BIND(ctx);
    if (nsteps == 0) return MM_OK;
    long K = checkpoint_every > 0 ? checkpoint_every : (long)std::ceil(std::sqrt((double)nsteps));
    if (K > nsteps) K = nsteps;
    const long nchk = (nsteps + K - 1) / K;
    const size_t e = ctx->prec == MM_F64 ? sizeof(double) : sizeof(float);
    const size_t v = 3 * (size_t)ctx->N * e;
    char* chk = nullptr;
    char* seg = nullptr;
    if (cudaMalloc((void**)&chk, v * nchk) != cudaSuccess || cudaMalloc((void**)&seg, v * K) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(chk);
        cudaFree(seg);
        return fail(ctx, MM_ERR_NOMEM, "checkpoint store of %ld + %ld states does not fit", nchk, K);
    }
    int rc = MM_OK;
    auto cp = [&](void* dst, const void* src) {
        if (rc == MM_OK) {
            cudaError_t ce = cudaMemcpyAsync(dst, src, v, cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce != cudaSuccess) rc = fail(ctx, MM_ERR_CUDA, "copy: %s", cudaGetErrorString(ce));
        }
    };
    // forward sweep: keep the state at the start of every segment
    rc = ctl_reset_push(ctx, 0.0, dt, INFINITY, 1.0);
    cp(seg, m0);
    for (long c = 0; c < nchk && rc == MM_OK; ++c) {
        cp(chk + c * v, seg);
        const long len = std::min(K, nsteps - c * K);
        if (rc == MM_OK && c + 1 < nchk) rc = rk4_steps(ctx, seg, len);
    }
    // the forward record of one segment (10 states per step) when it fits
    // the tape budget; otherwise each step VJP recomputes its stages
    char* tape = nullptr;
    if ((size_t)10 * v * (size_t)K <= kTapeBudget && cudaMalloc((void**)&tape, (size_t)10 * v * (size_t)K) != cudaSuccess) {
        cudaGetLastError();
        tape = nullptr;
    }
    auto tape_of = [&](long j) {
        StepTape t;
        char* b = tape + (size_t)j * 10 * v;
        for (int q = 0; q < 3; ++q) t.X[q] = b + q * v;
        for (int q = 0; q < 4; ++q) t.H[q] = b + (3 + q) * v;
        for (int q = 0; q < 3; ++q) t.k[q] = b + (7 + q) * v;
        return t;
    };
    // reverse sweep: replay each segment from its checkpoint, then pull lam
    // back through its steps (dt stays in the control block throughout)
    for (long c = nchk - 1; c >= 0 && rc == MM_OK; --c) {
        const long len = std::min(K, nsteps - c * K);
        cp(seg, chk + c * v);
        if (tape) {
            for (long j = 0; j < len && rc == MM_OK; ++j)
                rc = rk4_step_record(ctx, seg + j * v, j + 1 < len ? seg + (j + 1) * v : nullptr, tape_of(j));
        } else {
            for (long j = 1; j < len && rc == MM_OK; ++j) {
                cp(seg + j * v, seg + (j - 1) * v);
                if (rc == MM_OK) rc = rk4_steps(ctx, seg + j * v, 1);
            }
        }
        for (long j = len - 1; j >= 0 && rc == MM_OK; --j) {
            StepTape t;
            const StepTape* tp = nullptr;
            if (tape) {
                t = tape_of(j);
                tp = &t;
            }
            if (ctx->prec == MM_F64)
                rc = step_vjp<double>(ctx, (const double*)(seg + j * v), dt, (double*)lam, (double*)gMs, tp, false);
            else
                rc = step_vjp<float>(ctx, (const float*)(seg + j * v), dt, (float*)lam, (float*)gMs, tp, false);
        }
    }
    if (rc == MM_OK) rc = status_check(ctx);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tape);
    cudaFree(chk);
    cudaFree(seg);
    return rc;
}

}  // extern "C"
