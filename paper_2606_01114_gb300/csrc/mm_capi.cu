// C ABI entry points (include/mm.h): context lifetime, host-side sequencing
// of the Runge-Kutta stages and of relax(), scalar read-back, state files.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <limits>
#include <new>
#include <vector>

#include "mm_internal.cuh"

namespace mm {
// mm_exchange.cu: four-cell FP32 field kernels for uniform material (*done
// false when the context does not qualify)
int field4(mm_ctx* ctx, const void* m, const void* Hd, void* H, bool effective, bool* done);
}  // namespace mm

namespace mm {

static thread_local std::string g_init_error;

int fail(mm_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::string msg = std::string(err_name(code)) + ": " + buf;
    if (ctx) ctx->err = msg;
    else g_init_error = msg;
    return code;
}

const char* err_name(int code) {
    switch (code) {
        case MM_OK: return "ok";
        case MM_ERR_INVALID_ARG: return "invalid argument";
        case MM_ERR_CUDA: return "CUDA error";
        case MM_ERR_NONFINITE: return "non-finite value";
        case MM_ERR_DT_UNDERFLOW: return "time step underflow";
        case MM_ERR_NOT_CONVERGED: return "not converged";
        case MM_ERR_TIMEOUT: return "timeout";
        case MM_ERR_NOMEM: return "out of device memory";
        default: return "error";
    }
}

void harvest_timing(mm_ctx* ctx) {
    if (ctx->ev_used == 0) return;
    cudaStreamSynchronize(ctx->stream);
    for (size_t i = 0; i < ctx->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]) == cudaSuccess) {
            ctx->kt_ms[ctx->ev_kind[i]] += ms;
        }
    }
    cudaGetLastError();
    ctx->ev_used = 0;
}

// Every launch of a class is counted while timing is on; the classes in the
// mask are also bracketed by events (their device time is summed).
KernelTimer::KernelTimer(mm_ctx* c, int kind) : ctx(c), slot(0), on(((c->timing >> kind) & 1u) != 0) {
    if (c->timing) c->kt_n[kind] += 1;
    if (!on) return;
    if (ctx->ev_used >= 16384) harvest_timing(ctx);
    if (2 * (ctx->ev_used + 1) > ctx->ev_pool.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            cudaGetLastError();
            on = false;
            return;
        }
        ctx->ev_pool.push_back(a);
        ctx->ev_pool.push_back(b);
        ctx->ev_kind.push_back(0);
    }
    slot = ctx->ev_used++;
    ctx->ev_kind[slot] = kind;
    cudaEventRecord(ctx->ev_pool[2 * slot], ctx->stream);
}

KernelTimer::~KernelTimer() {
    if (on) cudaEventRecord(ctx->ev_pool[2 * slot + 1], ctx->stream);
}

namespace {

// nx, ny: any size up to 512 (powers of two take the fast passes, other
// sizes a direct DFT); nz: 1 or a power of two (the z pass is radix-2)
bool valid_n(int n) { return n >= 1 && n <= 512; }
bool valid_nz(int n) { return valid_n(n) && (n & (n - 1)) == 0; }
bool valid_len(double d) { return std::isfinite(d) && d > 0.0; }

size_t elem(const mm_ctx* ctx) { return ctx->prec == MM_F64 ? sizeof(double) : sizeof(float); }

void free_all(mm_ctx* ctx) {
    void* ptrs[] = {ctx->Ms_cell, ctx->A_cell, ctx->kern, ctx->bufA, ctx->bufB, ctx->Hd, ctx->Hs_field,
                    ctx->m0, ctx->ms[0], ctx->ms[1], ctx->mnext, ctx->kptrs, ctx->ctl, ctx->tw.f64, ctx->tw.f32,
                    ctx->tw.ff, ctx->kern_ff, ctx->adj, ctx->m_stage, ctx->kern_f4, ctx->tw_f4,
                    ctx->blue_x.chirp, ctx->blue_x.filt, ctx->blue_x.tw, ctx->blue_y.chirp, ctx->blue_y.filt,
                    ctx->blue_y.tw, ctx->blue_x.chirp32, ctx->blue_x.filt32, ctx->blue_x.tw32, ctx->blue_y.chirp32,
                    ctx->blue_y.filt32, ctx->blue_y.tw32};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (void* p : ctx->k)
        if (p) cudaFree(p);
    if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
    free(ctx->newell_host);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    ctx->ev_pool.clear();
}

// exp(-2 pi i m / L) for m < L, computed in long double and rounded
void twiddles(int L, std::vector<double>& out) {
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int m = 0; m < L; ++m) {
        long double a = 2.0L * pi * (long double)m / (long double)L;
        out.push_back((double)cosl(a));
        out.push_back((double)-sinl(a));
    }
}

int make_tables(mm_ctx* ctx) {
    std::vector<double> t;
    ctx->tw.off_lx = 0;
    twiddles(ctx->Lx, t);
    ctx->tw.off_px = (long)t.size() / 2;
    twiddles(ctx->Px, t);
    ctx->tw.off_py = (long)t.size() / 2;
    twiddles(ctx->Py, t);
    ctx->tw.off_pz = (long)t.size() / 2;
    twiddles(ctx->Pz, t);
    MM_CUDA_CHECK(ctx, cudaMalloc(&ctx->tw.f64, t.size() * sizeof(double)));
    MM_CUDA_CHECK(ctx, cudaMemcpy(ctx->tw.f64, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (ctx->prec == MM_F32) {
        std::vector<float> f(t.begin(), t.end());
        MM_CUDA_CHECK(ctx, cudaMalloc(&ctx->tw.f32, f.size() * sizeof(float)));
        MM_CUDA_CHECK(ctx, cudaMemcpy(ctx->tw.f32, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return MM_OK;
}

int alloc(mm_ctx* ctx, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? MM_ERR_NOMEM : MM_ERR_CUDA, "cudaMalloc of %zu bytes failed: %s",
                    bytes, cudaGetErrorString(e));
    }
    return MM_OK;
}

int push_ctl(mm_ctx* ctx) {
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(ctx->ctl, ctx->ctl_host, sizeof(Control), cudaMemcpyHostToDevice, ctx->stream));
    return MM_OK;
}
int pull_ctl(mm_ctx* ctx) {
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}
// wait for the stream before the host mirror is rewritten
int sync(mm_ctx* ctx) {
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

void reset_ctl(Control* c, double t, double dt, double t_max, double tol) {
    memset(c, 0, sizeof(Control));
    c->t = t;
    c->dt = dt;
    c->dt_next = dt;
    c->t_max = t_max;
    c->tol = tol;
}

// demag field of a stage state: the exact convolution, or the surrogate
// (output scaled by Ms) when one is attached for this window
int stage_field(mm_ctx* ctx, const void* m_in) {
    if (ctx->stage_surrogate) {
        ++ctx->surrogate_evals;
        return mm_fno_forward(ctx->stage_surrogate, m_in, ctx->Hd, 1);
    }
    ++ctx->exact_evals;
    return demag_apply(ctx, m_in, ctx->Hd);
}

// one trial step from m (RK4 writes m in place; RKF45 writes mnext and commits)
int trial(mm_ctx* ctx, void* m, int method) {
    const int S = method == MM_RK4 ? 4 : 6;
    int rc;
    for (int s = 0; s < S; ++s) {
        const void* m_in = s == 0 ? m : ctx->ms[s % 2];
        void* m_out = s < S - 1 ? ctx->ms[(s + 1) % 2] : (method == MM_RK4 ? m : ctx->mnext);
        if ((rc = stage_field(ctx, m_in))) return rc;
        if ((rc = rk_stage(ctx, method, s, m_in, m, m_out))) return rc;
    }
    if ((rc = rk_controller(ctx, method))) return rc;
    if (method == MM_RKF45 && (rc = rk_commit(ctx, m))) return rc;
    return MM_OK;
}

int device_status(mm_ctx* ctx) {
    int st = ctx->ctl_host->status;
    if (st == MM_ERR_NONFINITE) return fail(ctx, st, "NaN or Inf in the magnetisation");
    if (st == MM_ERR_DT_UNDERFLOW) return fail(ctx, st, "RKF45 step fell below 1e-20 s");
    if (st == MM_ERR_TIMEOUT) return fail(ctx, st, "a bounded device wait (TMA-fed demag pass) gave up");
    if (st) return fail(ctx, st, "device status %d", st);
    return MM_OK;
}

}  // namespace

int ctl_reset_push(mm_ctx* ctx, double t, double dt, double t_max, double tol) {
    int rc = sync(ctx);
    if (rc) return rc;
    reset_ctl(ctx->ctl_host, t, dt, t_max, tol);
    return push_ctl(ctx);
}
int ctl_pull(mm_ctx* ctx) { return pull_ctl(ctx); }

}  // namespace mm

using namespace mm;

extern "C" {

int mm_init_mesh(mm_ctx** out, int nx, int ny, int nz, double dx, double dy, double dz, int precision,
                 void* stream) {
    if (!out) return fail(nullptr, MM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_n(nx) || !valid_n(ny) || !valid_nz(nz))
        return fail(nullptr, MM_ERR_INVALID_ARG,
                    "mesh %dx%dx%d: nx, ny in 1..512, nz 1 or a power of two <= 512", nx, ny, nz);
    if (!valid_len(dx) || !valid_len(dy) || !valid_len(dz))
        return fail(nullptr, MM_ERR_INVALID_ARG, "cell size must be finite and > 0");
    if (precision != MM_F32 && precision != MM_F64) return fail(nullptr, MM_ERR_INVALID_ARG, "bad precision");
    mm_ctx* ctx = new (std::nothrow) mm_ctx();
    if (!ctx) return fail(nullptr, MM_ERR_NOMEM, "host allocation failed");
    ctx->nx = nx;
    ctx->ny = ny;
    ctx->nz = nz;
    ctx->dx = dx;
    ctx->dy = dy;
    ctx->dz = dz;
    ctx->prec = precision;
    ctx->stream = (cudaStream_t)stream;
    {
        int dev = 0;
        cudaError_t ce = stream ? cudaStreamGetDevice(ctx->stream, &dev) : cudaGetDevice(&dev);
        if (ce == cudaSuccess) ce = cudaSetDevice(dev);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return fail(nullptr, MM_ERR_CUDA, "cannot select the stream's device: %s", cudaGetErrorString(ce));
        }
        ctx->device = dev;
    }
    ctx->N = (long)nx * ny * nz;
    ctx->Px = nx > 1 ? 2 * nx : 1;
    ctx->Py = ny > 1 ? 2 * ny : 1;
    ctx->Pz = nz > 1 ? 2 * nz : 1;
    ctx->Lx = nx > 1 ? nx : 1;
    ctx->Hx = nx > 1 ? nx + 1 : 1;
    ctx->Hs = (ctx->Hx + 15) / 16 * 16;
    ctx->Py2 = ctx->Py / 2 + 1;
    ctx->Pz2 = ctx->Pz / 2 + 1;
    ctx->Ms = 8e5;
    ctx->A = 1.3e-11;
    ctx->alpha = 0.02;
    ctx->Ku = 0.0;
    ctx->u[0] = 0.0;
    ctx->u[1] = 0.0;
    ctx->u[2] = 1.0;
    const size_t e = elem(ctx);
    const size_t v3 = 3 * (size_t)ctx->N * e;
    int rc = MM_OK;
    auto A = [&](void** p, size_t b) {
        if (rc == MM_OK) rc = alloc(ctx, p, b);
    };
    A(&ctx->kern, 6 * (size_t)ctx->Pz2 * ctx->Py2 * ctx->Hs * e);
    A(&ctx->bufA, 3 * (size_t)nz * ny * ctx->Hs * 2 * e);
    A(&ctx->bufB, 3 * (size_t)nz * ctx->Py * ctx->Hs * 2 * e);
    A(&ctx->Hd, v3);
    A(&ctx->Hs_field, v3);
    A(&ctx->ms[0], v3);
    A(&ctx->ms[1], v3);
    A(&ctx->mnext, v3);
    for (int s = 0; s < 6; ++s) A(&ctx->k[s], v3);
    A(&ctx->kptrs, 6 * sizeof(void*));
    A(&ctx->Ms_cell, (size_t)ctx->N * e);
    A(&ctx->A_cell, (size_t)ctx->N * e);
    A((void**)&ctx->ctl, sizeof(Control));
    if (rc == MM_OK && cudaMallocHost((void**)&ctx->ctl_host, sizeof(Control)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(ctx, MM_ERR_NOMEM, "pinned allocation failed");
    }
    if (rc == MM_OK) {
        ctx->newell_host = (double*)malloc(sizeof(double) * 6 * ctx->N);
        if (!ctx->newell_host) rc = fail(ctx, MM_ERR_NOMEM, "host allocation failed");
    }
    if (rc == MM_OK) {
        cudaError_t ce = cudaMemcpy(ctx->kptrs, ctx->k, 6 * sizeof(void*), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) rc = fail(ctx, MM_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(ce));
    }
    if (rc == MM_OK) rc = make_tables(ctx);
    if (rc == MM_OK) rc = blue_prepare(ctx);
    if (rc == MM_OK) {
        reset_ctl(ctx->ctl_host, 0.0, 1e-14, std::numeric_limits<double>::infinity(), 1e-5);
        rc = push_ctl(ctx);
    }
    if (rc == MM_OK) rc = demag_setup(ctx);
    if (rc == MM_OK) rc = sync(ctx);
    if (rc != MM_OK) {
        g_init_error = ctx->err;
        free_all(ctx);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return MM_OK;
}

int mm_set_stream(mm_ctx* ctx, void* stream) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (stream) {
        int dev = -1;
        MM_CUDA_CHECK(ctx, cudaStreamGetDevice((cudaStream_t)stream, &dev));
        if (dev != ctx->device) return fail(ctx, MM_ERR_INVALID_ARG, "stream is on device %d, context on %d", dev, ctx->device);
    }
    ctx->stream = (cudaStream_t)stream;
    return MM_OK;
}

int mm_set_material(mm_ctx* ctx, double Ms, double A, double alpha, double Ku, const double u_anis[3]) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!(std::isfinite(Ms) && Ms >= 0) || !(std::isfinite(A) && A >= 0) || !(std::isfinite(alpha) && alpha >= 0) ||
        !std::isfinite(Ku))
        return fail(ctx, MM_ERR_INVALID_ARG, "material values must be finite, Ms, A, alpha >= 0");
    double u[3] = {0.0, 0.0, 1.0};
    if (u_anis) {
        double n = std::sqrt(u_anis[0] * u_anis[0] + u_anis[1] * u_anis[1] + u_anis[2] * u_anis[2]);
        if (!(n > 0) || !std::isfinite(n)) return fail(ctx, MM_ERR_INVALID_ARG, "anisotropy axis must be non-zero");
        for (int c = 0; c < 3; ++c) u[c] = u_anis[c] / n;
    }
    ctx->Ms = Ms;
    ctx->A = A;
    ctx->alpha = alpha;
    ctx->Ku = Ku;
    for (int c = 0; c < 3; ++c) ctx->u[c] = u[c];
    return MM_OK;
}

int mm_set_material_fields(mm_ctx* ctx, const void* Ms_cell, const void* A_cell) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    const size_t b = (size_t)ctx->N * elem(ctx);
    if (Ms_cell) MM_CUDA_CHECK(ctx, cudaMemcpyAsync(ctx->Ms_cell, Ms_cell, b, cudaMemcpyDeviceToDevice, ctx->stream));
    if (A_cell) MM_CUDA_CHECK(ctx, cudaMemcpyAsync(ctx->A_cell, A_cell, b, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->has_Ms_cell = Ms_cell != nullptr;
    ctx->has_A_cell = A_cell != nullptr;
    return MM_OK;
}

int mm_set_external_field(mm_ctx* ctx, double hx, double hy, double hz) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!std::isfinite(hx) || !std::isfinite(hy) || !std::isfinite(hz))
        return fail(ctx, MM_ERR_INVALID_ARG, "external field must be finite");
    ctx->hext[0] = hx;
    ctx->hext[1] = hy;
    ctx->hext[2] = hz;
    return MM_OK;
}

int mm_demag_field(mm_ctx* ctx, const void* m, void* H) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !H) return fail(ctx, MM_ERR_INVALID_ARG, "m and H must be device pointers");
    return demag_apply(ctx, m, H);
}

int mm_exchange_field(mm_ctx* ctx, const void* m, void* H) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !H) return fail(ctx, MM_ERR_INVALID_ARG, "m and H must be device pointers");
    bool done = false;
    int rc = field4(ctx, m, nullptr, H, false, &done);
    if (rc || done) return rc;
    return field_exchange(ctx, m, H);
}

int mm_effective_field(mm_ctx* ctx, const void* m, void* H) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !H) return fail(ctx, MM_ERR_INVALID_ARG, "m and H must be device pointers");
    int rc = demag_apply(ctx, m, ctx->Hd);
    if (rc) return rc;
    bool done = false;
    rc = field4(ctx, m, ctx->Hd, H, true, &done);
    if (rc || done) return rc;
    return field_effective(ctx, m, ctx->Hd, H);
}

int mm_llg_step(mm_ctx* ctx, void* m, double* t, double* dt, int method, double tol, double* err_out) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !t || !dt) return fail(ctx, MM_ERR_INVALID_ARG, "m, t, dt must not be NULL");
    if (method != MM_RK4 && method != MM_RKF45) return fail(ctx, MM_ERR_INVALID_ARG, "bad method %d", method);
    if (!(std::isfinite(*dt) && *dt > 0) || !std::isfinite(*t)) return fail(ctx, MM_ERR_INVALID_ARG, "dt must be > 0");
    if (method == MM_RKF45 && !(std::isfinite(tol) && tol > 0))
        return fail(ctx, MM_ERR_INVALID_ARG, "tol must be > 0");
    int rc;
    if ((rc = sync(ctx))) return rc;
    reset_ctl(ctx->ctl_host, *t, *dt, std::numeric_limits<double>::infinity(), tol);
    if ((rc = push_ctl(ctx))) return rc;
    if ((rc = check_finite_launch(ctx, m))) return rc;
    for (int attempt = 0; attempt < 200; ++attempt) {
        if ((rc = trial(ctx, m, method))) return rc;
        if ((rc = pull_ctl(ctx))) return rc;
        if ((rc = device_status(ctx))) return rc;
        if (ctx->ctl_host->accepted) {
            *t = ctx->ctl_host->t;
            *dt = method == MM_RK4 ? *dt : ctx->ctl_host->dt;
            if (err_out) *err_out = method == MM_RK4 ? 0.0 : ctx->ctl_host->last_err;
            return MM_OK;
        }
    }
    return fail(ctx, MM_ERR_DT_UNDERFLOW, "RKF45 rejected 200 trials in a row");
}

int mm_llg_step_host(mm_ctx* ctx, void* m_host, double* t, double* dt, int method, double tol, double* err_out) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m_host) return fail(ctx, MM_ERR_INVALID_ARG, "m_host must not be NULL");
    const size_t bytes = 3 * (size_t)ctx->N * elem(ctx);
    int rc;
    if (!ctx->m_stage && (rc = alloc(ctx, &ctx->m_stage, bytes))) return rc;
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(ctx->m_stage, m_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = mm_llg_step(ctx, ctx->m_stage, t, dt, method, tol, err_out))) return rc;
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(m_host, ctx->m_stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_kspace_product(mm_ctx* ctx, void* spectrum) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!spectrum) return fail(ctx, MM_ERR_INVALID_ARG, "spectrum must be a device pointer");
    return demag_kspace_product(ctx, spectrum);
}

int mm_relax(mm_ctx* ctx, void* m, double t_max, double torque_tol, long max_steps, double* t_out, long* steps_out) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m) return fail(ctx, MM_ERR_INVALID_ARG, "m must not be NULL");
    if (!(t_max > 0) || !(torque_tol >= 0) || max_steps < 0)
        return fail(ctx, MM_ERR_INVALID_ARG, "t_max > 0, torque_tol >= 0, max_steps >= 0 required");
    int rc;
    if ((rc = sync(ctx))) return rc;
    reset_ctl(ctx->ctl_host, 0.0, std::fmin(1e-14, t_max), t_max, 1e-5);
    if ((rc = push_ctl(ctx))) return rc;
    if ((rc = check_finite_launch(ctx, m))) return rc;
    const int kCheck = 10;
    long attempts = 0;
    const long max_attempts = 20 * (max_steps + 10);
    while (true) {
        // torque of the current state
        MM_CUDA_CHECK(ctx, cudaMemsetAsync(&ctx->ctl->torque_bits, 0, sizeof(unsigned long long), ctx->stream));
        if ((rc = demag_apply(ctx, m, ctx->Hd))) return rc;
        if ((rc = torque_launch(ctx, m, ctx->Hd))) return rc;
        if ((rc = pull_ctl(ctx))) return rc;
        if ((rc = device_status(ctx))) return rc;
        const Control* c = ctx->ctl_host;
        double tq;
        unsigned long long bits = c->torque_bits;
        memcpy(&tq, &bits, sizeof(tq));
        if (t_out) *t_out = c->t;
        if (steps_out) *steps_out = (long)c->steps;
        if (tq <= torque_tol || c->done) return MM_OK;
        if (c->steps >= max_steps || attempts >= max_attempts)
            return fail(ctx, MM_ERR_NOT_CONVERGED, "relax stopped after %lld steps, torque %.3e", (long long)c->steps, tq);
        // each trial accepts at most one step: a batch no longer than the
        // steps still allowed stops relax at exactly max_steps
        const long room = max_steps - (long)c->steps;
        const int batch = room < kCheck ? (int)room : kCheck;
        for (int k = 0; k < batch; ++k, ++attempts)
            if ((rc = trial(ctx, m, MM_RKF45))) return rc;
    }
}

int mm_set_dmi(mm_ctx* ctx, double D, int type) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!std::isfinite(D) || (type != MM_DMI_INTERFACIAL && type != MM_DMI_BULK))
        return fail(ctx, MM_ERR_INVALID_ARG, "DMI: finite D and type MM_DMI_INTERFACIAL or MM_DMI_BULK required");
    ctx->D = D;
    ctx->dmi_type = type;
    return MM_OK;
}

int mm_set_stt(mm_ctx* ctx, double J, double P, double Lambda, double eps_prime, const double p[3], double d) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (J == 0.0) {
        ctx->stt_on = 0;
        return MM_OK;
    }
    if (!p || !std::isfinite(J) || !std::isfinite(P) || !(Lambda >= 1.0) || !std::isfinite(eps_prime) ||
        !std::isfinite(d))
        return fail(ctx, MM_ERR_INVALID_ARG, "STT: finite J, P, eps', Lambda >= 1 and a polarisation vector required");
    const double n = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if (!(n > 0) || !std::isfinite(n)) return fail(ctx, MM_ERR_INVALID_ARG, "STT: polarisation vector must be non-zero");
    ctx->stt_on = 1;
    ctx->stt_J = J;
    ctx->stt_P = P;
    ctx->stt_L = Lambda;
    ctx->stt_eps2 = eps_prime;
    for (int c = 0; c < 3; ++c) ctx->stt_p[c] = p[c] / n;
    ctx->stt_d = d > 0 ? d : ctx->nz * ctx->dz;
    return MM_OK;
}

int mm_minimize_bb(mm_ctx* ctx, void* m, double torque_tol, long max_iter, long* iters_out) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m) return fail(ctx, MM_ERR_INVALID_ARG, "m must not be NULL");
    if (!(torque_tol >= 0) || max_iter < 0) return fail(ctx, MM_ERR_INVALID_ARG, "torque_tol >= 0, max_iter >= 0 required");
    int rc;
    if ((rc = sync(ctx))) return rc;
    reset_ctl(ctx->ctl_host, 0.0, 0.0, 0.0, 0.0);
    if ((rc = push_ctl(ctx))) return rc;
    if ((rc = check_finite_launch(ctx, m))) return rc;
    // slope buffers of the integrator serve as g (two, alternating) and m_prev
    void* gb[2] = {ctx->k[0], ctx->k[1]};
    void* m_prev = ctx->k[2];
    const int kCheck = 10;
    for (long it = 0;; ++it) {
        if ((rc = demag_apply(ctx, m, ctx->Hd))) return rc;
        if ((rc = bb_iteration(ctx, m, gb[it & 1], gb[(it + 1) & 1], m_prev, it > 0, torque_tol, max_iter))) return rc;
        if ((it + 1) % kCheck == 0 || it >= max_iter) {
            if ((rc = pull_ctl(ctx))) return rc;
            if ((rc = device_status(ctx))) return rc;
            if (ctx->ctl_host->done) break;
        }
    }
    const Control* c = ctx->ctl_host;
    if (iters_out) *iters_out = (long)c->steps;
    double tq;
    unsigned long long bits = c->torque_bits;
    memcpy(&tq, &bits, sizeof(tq));
    if (!(tq <= torque_tol))
        return fail(ctx, MM_ERR_NOT_CONVERGED, "minimiser stopped after %lld steps, torque %.3e", (long long)c->steps, tq);
    return MM_OK;
}

int mm_relax_surrogate(mm_ctx* ctx, mm_fno* f, void* m, double t_max, double torque_tol, long max_steps,
                       int k_exact, double bound, double torque_exact, double* t_out, long* steps_out, long* stats) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!f || !m || k_exact < 1 || !(t_max > 0) || !(torque_tol >= 0) || max_steps < 0 || !(bound >= 0))
        return fail(ctx, MM_ERR_INVALID_ARG, "surrogate, m, k_exact >= 1, t_max > 0, bounds >= 0 required");
    if (ctx->prec != MM_F32 || ctx->nz != 1 || ctx->has_Ms_cell)
        return fail(ctx, MM_ERR_INVALID_ARG, "the surrogate serves MM_F32 films (nz = 1) of uniform Ms");
    int fnx, fny;
    fno_grid(f, &fnx, &fny);
    if (fnx != ctx->nx || fny != ctx->ny) return fail(ctx, MM_ERR_INVALID_ARG, "surrogate grid differs from the mesh");
    MM_BIND(ctx);
    int rc;
    if ((rc = sync(ctx))) return rc;
    if ((rc = mm_fno_set_output_scale(f, ctx->Ms))) return rc;
    const cudaStream_t fno_stream = fno_swap_stream(f, ctx->stream);
    reset_ctl(ctx->ctl_host, 0.0, std::fmin(1e-14, t_max), t_max, 1e-5);
    if ((rc = push_ctl(ctx))) return rc;
    if ((rc = check_finite_launch(ctx, m))) return rc;
    long exact0 = ctx->exact_evals, sur0 = ctx->surrogate_evals, fallbacks = 0, attempts = 0;
    const long max_attempts = 20 * (max_steps + 10);
    // after a failed residual check the next check waits 1, 2, 4, ... windows
    // (at most 64), so a surrogate that does not fit the state costs little
    long skip = 0, backoff = 1;
    rc = MM_OK;
    while (rc == MM_OK) {
        // window start: exact field and torque, then (when due) the surrogate's residual
        MM_CUDA_CHECK(ctx, cudaMemsetAsync(&ctx->ctl->torque_bits, 0, sizeof(unsigned long long), ctx->stream));
        ++ctx->exact_evals;
        if ((rc = demag_apply(ctx, m, ctx->Hs_field))) break;
        if ((rc = torque_launch(ctx, m, ctx->Hs_field))) break;
        if ((rc = pull_ctl(ctx))) break;
        if ((rc = device_status(ctx))) break;
        const Control* c = ctx->ctl_host;
        double tq;
        unsigned long long bits = c->torque_bits;
        memcpy(&tq, &bits, sizeof(tq));
        if (t_out) *t_out = c->t;
        if (steps_out) *steps_out = (long)c->steps;
        if (tq <= torque_tol || c->done) break;
        if (c->steps >= max_steps || attempts >= max_attempts) {
            rc = fail(ctx, MM_ERR_NOT_CONVERGED, "surrogate relax stopped after %lld steps, torque %.3e",
                      (long long)c->steps, tq);
            break;
        }
        const long steps_now = (long)c->steps;
        bool use = false;
        if (tq > torque_exact) {   // at or below torque_exact: the final approach is exact
            if (skip > 0) {
                --skip;
            } else {
                ++ctx->surrogate_evals;
                if ((rc = mm_fno_forward(f, m, ctx->Hd, 1))) break;
                double loss = 0.0;
                if ((rc = mm_fno_loss(f, ctx->Hd, ctx->Hs_field, nullptr, 1, &loss))) break;
                use = std::sqrt(loss) <= bound;
                if (use) {
                    backoff = 1;
                } else {
                    ++fallbacks;
                    skip = backoff;
                    backoff = std::min(2 * backoff, 64L);
                }
            }
        }
        ctx->stage_surrogate = use ? f : nullptr;
        const long target = steps_now + k_exact;
        for (int k = 0; k < 4 * k_exact && rc == MM_OK; ++k, ++attempts) {
            rc = trial(ctx, m, MM_RKF45);
            if (rc == MM_OK && (k + 1) % k_exact == 0) {
                if ((rc = pull_ctl(ctx))) break;
                if (ctx->ctl_host->steps >= target || ctx->ctl_host->done || ctx->ctl_host->status) break;
            }
        }
        ctx->stage_surrogate = nullptr;
    }
    ctx->stage_surrogate = nullptr;
    fno_swap_stream(f, fno_stream);
    mm_fno_set_output_scale(f, 1.0);
    if (stats) {
        stats[0] = ctx->exact_evals - exact0;
        stats[1] = ctx->surrogate_evals - sur0;
        stats[2] = fallbacks;
    }
    return rc;
}

int mm_energy(mm_ctx* ctx, const void* m, double E_out[5]) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !E_out) return fail(ctx, MM_ERR_INVALID_ARG, "m and E_out must not be NULL");
    int rc;
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->ctl->energy, 0, 5 * sizeof(double), ctx->stream));
    if ((rc = demag_apply(ctx, m, ctx->Hd))) return rc;
    if ((rc = energy_launch(ctx, m, ctx->Hd))) return rc;
    if ((rc = pull_ctl(ctx))) return rc;
    for (int i = 0; i < 5; ++i) E_out[i] = ctx->ctl_host->energy[i];
    return MM_OK;
}

int mm_max_torque(mm_ctx* ctx, const void* m, double* out) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !out) return fail(ctx, MM_ERR_INVALID_ARG, "m and out must not be NULL");
    int rc;
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(&ctx->ctl->torque_bits, 0, sizeof(unsigned long long), ctx->stream));
    if ((rc = demag_apply(ctx, m, ctx->Hd))) return rc;
    if ((rc = torque_launch(ctx, m, ctx->Hd))) return rc;
    if ((rc = pull_ctl(ctx))) return rc;
    unsigned long long bits = ctx->ctl_host->torque_bits;
    memcpy(out, &bits, sizeof(double));
    return MM_OK;
}

int mm_newell_tensor(mm_ctx* ctx, double* host_out) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (!host_out) return fail(ctx, MM_ERR_INVALID_ARG, "host_out is NULL");
    memcpy(host_out, ctx->newell_host, sizeof(double) * 6 * ctx->N);
    return MM_OK;
}

struct StateHeader {
    char magic[8];
    int nx, ny, nz, prec;
    double t, dt;
};

int mm_save_state(mm_ctx* ctx, const void* m, double t, double dt, const char* path) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !path) return fail(ctx, MM_ERR_INVALID_ARG, "m and path must not be NULL");
    const size_t b = 3 * (size_t)ctx->N * elem(ctx);
    std::vector<char> buf(b);
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(buf.data(), m, b, cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    StateHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "MMGB300", 8);
    h.nx = ctx->nx;
    h.ny = ctx->ny;
    h.nz = ctx->nz;
    h.prec = ctx->prec;
    h.t = t;
    h.dt = dt;
    FILE* f = fopen(path, "wb");
    if (!f) return fail(ctx, MM_ERR_INVALID_ARG, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 1, b, f) == b;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, MM_ERR_INVALID_ARG, "write to %s failed", path);
    return MM_OK;
}

int mm_load_state(mm_ctx* ctx, void* m, double* t, double* dt, const char* path) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    MM_BIND(ctx);
    if (!m || !path) return fail(ctx, MM_ERR_INVALID_ARG, "m and path must not be NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(ctx, MM_ERR_INVALID_ARG, "cannot open %s", path);
    StateHeader h;
    const size_t b = 3 * (size_t)ctx->N * elem(ctx);
    std::vector<char> buf(b);
    bool ok = fread(&h, sizeof(h), 1, f) == 1;
    ok = ok && memcmp(h.magic, "MMGB300", 8) == 0 && h.nx == ctx->nx && h.ny == ctx->ny && h.nz == ctx->nz &&
         h.prec == ctx->prec;
    ok = ok && fread(buf.data(), 1, b, f) == b;
    fclose(f);
    if (!ok) return fail(ctx, MM_ERR_INVALID_ARG, "%s is not a state file of this mesh and precision", path);
    MM_CUDA_CHECK(ctx, cudaMemcpyAsync(m, buf.data(), b, cudaMemcpyHostToDevice, ctx->stream));
    MM_CUDA_CHECK(ctx, cudaStreamSynchronize(ctx->stream));
    if (t) *t = h.t;
    if (dt) *dt = h.dt;
    return MM_OK;
}

void mm_destroy(mm_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

const char* mm_last_error(const mm_ctx* ctx) {
    if (!ctx) return g_init_error.c_str();
    return ctx->err.c_str();
}

long mm_kernel_launches(const mm_ctx* ctx) { return ctx ? ctx->launches : 0; }

int mm_enable_kernel_timing_mask(mm_ctx* ctx, unsigned classes) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (classes >> MM_K_COUNT) return fail(ctx, MM_ERR_INVALID_ARG, "timing mask 0x%x names no kernel class", classes);
    harvest_timing(ctx);
    for (int k = 0; k < MM_K_COUNT; ++k) {
        ctx->kt_ms[k] = 0.0;
        ctx->kt_n[k] = 0;
    }
    ctx->timing = classes;
    return MM_OK;
}

int mm_enable_kernel_timing(mm_ctx* ctx, int enable) {
    return mm_enable_kernel_timing_mask(ctx, enable ? (1u << MM_K_COUNT) - 1u : 0u);
}

int mm_kernel_time(mm_ctx* ctx, int kernel, double* total_ms, long* launches) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    if (kernel < 0 || kernel >= MM_K_COUNT) return fail(ctx, MM_ERR_INVALID_ARG, "bad kernel class %d", kernel);
    harvest_timing(ctx);
    if (total_ms) *total_ms = ctx->kt_ms[kernel];
    if (launches) *launches = ctx->kt_n[kernel];
    return MM_OK;
}

int mm_step_stats(const mm_ctx* ctx, long* accepted, long* rejected, double* t, double* dt) {
    if (!ctx) return fail(nullptr, MM_ERR_INVALID_ARG, "ctx is NULL");
    const Control* c = ctx->ctl_host;
    if (accepted) *accepted = (long)c->steps;
    if (rejected) *rejected = (long)c->rejects;
    if (t) *t = c->t;
    if (dt) *dt = c->dt;
    return MM_OK;
}

}  // extern "C"
