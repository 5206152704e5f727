// Internal declarations shared by the translation units of libmm_gb300.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mm.h"

namespace mm {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kMu0 = 4e-7 * kPi;
constexpr double kGamma = 2.2127615e5;   // mu0 * gamma_e, m / (A s)
constexpr double kHbar = 1.054571817e-34;   // J s
constexpr double kQe = 1.602176634e-19;     // C

// ---------------------------------------------------------------- complex
template <typename T> struct cx;
template <> struct cx<float> { using type = float2; };
template <> struct cx<double> { using type = double2; };

template <typename C> __host__ __device__ __forceinline__ C cmk(decltype(C{}.x) a, decltype(C{}.x) b) {
    C r; r.x = a; r.y = b; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(C{}.x) s) { return cmk<C>(a.x * s, a.y * s); }

// --------------------------------------------------------- device control
// One RKF45/RK4 control block per context, in device memory.
struct Control {
    double t;            // simulated time
    double dt;           // step of the trial in flight
    double dt_next;      // proposal after the controller ran
    double t_max;        // relax(): end time (inf for plain steps)
    double tol;          // RKF45 tolerance
    unsigned long long err_bits;     // max error of the trial (double bits, >= 0)
    unsigned long long torque_bits;  // max torque / Ms (double bits)
    double energy[5];    // demag, exchange, anisotropy, Zeeman, DMI
    double bb[3];        // minimiser: sums s.s, s.y, y.y
    int accepted;        // 1 if the last trial was accepted
    int status;          // 0 or an MM_ERR_* code raised on the device
    int done;            // relax(): t reached t_max
    int pad;
    double last_err;     // error of the last accepted RKF45 trial
    long long steps;     // accepted steps
    long long rejects;   // rejected trials
};

// --------------------------------------------------------------- context
struct Tables {
    // exp(-2 pi i m / L), m in [0, L), for L in {Lx, Px, Py, Pz}
    void* f64 = nullptr;   // double2
    void* f32 = nullptr;   // float2 (only for MM_F32 contexts)
    void* ff = nullptr;    // float-float copy of f64 (MM_FFT_FF on an MM_F64 context)
    long off_lx = 0, off_px = 0, off_py = 0, off_pz = 0;
};

// Bluestein (chirp-z) data of one padded axis whose length P is not a power
// of two: transforms of P points as a convolution of length M (the power of
// two >= 2P - 1).  Arrays at the context's precision (complex):
//   chirp[n] = exp(-i pi n^2 / P), n < P (DIR +1 uses its conjugate);
//   filt[d]  = FFT_M of b_d[j] = exp(-d i pi j^2 / P) on |j| < P (wrapped
//              mod M), scaled by 1/M, for d = -1 (index 0) and +1 (index 1);
//   tw[m]    = exp(-2 pi i m / M), m < M.
struct Blue {
    int P = 0, M = 0;
    void* chirp = nullptr;   // double2 (the Newell setup runs its passes in FP64)
    void* filt = nullptr;    // double2 [2][M]
    void* tw = nullptr;      // double2
    void* chirp32 = nullptr; // float2 copies for MM_F32 contexts
    void* filt32 = nullptr;
    void* tw32 = nullptr;
};

}  // namespace mm

struct mm_ctx {
    int nx, ny, nz;
    double dx, dy, dz;
    int prec;                 // MM_F32 / MM_F64
    int device;               // CUDA device of the stream
    cudaStream_t stream;
    long N;                   // cells
    int Px, Py, Pz;           // padded FFT sizes (2n, or 1 when n == 1)
    int Lx;                   // complex length of the packed real x transform (Px/2, or 1)
    int Hx;                   // kept x frequencies (nx + 1, or 1)
    int Hs;                   // row stride of k-space arrays (Hx rounded up to 16)
    int Py2, Pz2;             // Py/2+1, Pz/2+1: stored kernel octant extents
    int fft_mode;             // 0 plain passes, MM_TC_TF32 / MM_TC_BF16: tensor-core y passes (FP32),
                              // MM_FFT_FF: float-float passes (FP64)
    mm_fno* stage_surrogate;  // set inside mm_relax_surrogate while a window uses the surrogate
    long surrogate_evals, exact_evals;   // demag evaluations of either kind (surrogate relax statistics)

    // material
    double Ms, A, alpha, Ku, u[3], hext[3];
    double D;                 // DMI constant (J/m^2)
    int dmi_type;             // 0 none, MM_DMI_INTERFACIAL, MM_DMI_BULK
    // Slonczewski torque: on, J (A/m^2), P, Lambda, eps', unit p, free-layer thickness d (m)
    int stt_on;
    double stt_J, stt_P, stt_L, stt_eps2, stt_p[3], stt_d;
    bool has_Ms_cell, has_A_cell;
    void* Ms_cell;            // [N] path precision (allocated always; filled when used)
    void* A_cell;

    // buffers (path precision T; complex = 2T)
    void* kern;               // [6][Pz2][Py2][Hs] real k-space Newell octant
    void* kern_ff;            // float-float copy of kern (MM_FFT_FF), or NULL
    void* kern_f4;            // octant re-laid out per kx plane for MM_FFT_F4, or NULL
    void* tw_f4;              // twiddles of the fused MM_FFT_F4 pass, or NULL
    void* bufA;               // complex [3][nz][ny][Hs]
    void* bufB;               // complex [3][nz][Py][Hs]
    void* Hd;                 // [3][N] demag field of the current stage state
    void* Hs_field;           // [3][N] scratch field
    void* m0;                 // [3][N] internal copy of the state for relax
    void* ms[2];              // [3][N] trial states (ping-pong)
    void* mnext;              // [3][N] accepted-candidate state
    void* k[6];               // [3][N] RK stage slopes
    void* kptrs;              // device copy of k[0..5]
    void* adj;                // adjoint workspace (14 fields of [3][N]), allocated on first use
    void* m_stage;            // [3][N] device copy of a host state (mm_llg_step_host), allocated on first use
    mm::Control* ctl;         // device control block
    mm::Control* ctl_host;    // pinned host mirror
    double* newell_host;      // [6][nz][ny][nx] real-space tensor (host copy)
    mm::Tables tw;
    mm::Blue blue_x, blue_y;  // Bluestein data of Px and Py when they are not powers of two
    // TMA descriptors (CUtensorMap bytes) of the y passes' inputs, FP32
    // contexts with Py = 512 or 1024: [0] bufA as [3 nz][ny][Hs] complex,
    // [1] bufB as [3 nz][Py][Hs]; encoded on first use
    alignas(64) unsigned char ymap[2][128];
    int ymap_state;           // 0 not tried, 1 ready, -1 not available (register passes instead)
    int ymap_grid[2];         // persistent grids of the TMA-fed y forward [0] and inverse [1] passes
    int xtma_state;           // TMA-fed x inverse (nx = 512): 0 not tried, 1 ready, -1 not available
    int xtma_grid;            // its persistent grid

    long launches;
    std::string err;

    // per-kernel timing (mm_enable_kernel_timing)
    unsigned timing;                    // bit k: bracket launches of kernel class k with events
    std::vector<cudaEvent_t> ev_pool;   // pairs (start, stop)
    std::vector<int> ev_kind;           // kernel class of each pair
    size_t ev_used;                     // pairs recorded since the last harvest
    double kt_ms[MM_K_COUNT];
    long kt_n[MM_K_COUNT];
};

namespace mm {

// Set ctx->err and return code.
int fail(mm_ctx* ctx, int code, const char* fmt, ...);
const char* err_name(int code);

#define MM_CUDA_CHECK(ctx, call)                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return ::mm::fail((ctx), MM_ERR_CUDA, "%s failed: %s (%s:%d)", #call,      \
                              cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)

// make the context's device current for this thread (the library links its
// own CUDA runtime, whose current device is separate from the caller's)
#define MM_BIND(ctx)                                                                   \
    do {                                                                               \
        cudaError_t e_ = cudaSetDevice((ctx)->device);                                 \
        if (e_ != cudaSuccess)                                                         \
            return ::mm::fail((ctx), MM_ERR_CUDA, "cudaSetDevice(%d): %s", (ctx)->device, \
                              cudaGetErrorString(e_));                                 \
    } while (0)

#define MM_LAUNCH_CHECK(ctx)                                                           \
    do {                                                                               \
        (ctx)->launches++;                                                             \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess)                                                         \
            return ::mm::fail((ctx), MM_ERR_CUDA, "kernel launch failed: %s (%s:%d)",  \
                              cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)

// Brackets the launches in its scope with CUDA events when timing is on.
struct KernelTimer {
    mm_ctx* ctx;
    size_t slot;
    bool on;
    KernelTimer(mm_ctx* c, int kind);
    ~KernelTimer();
};

// Column transform geometry shared by the plain and tensor-core y passes:
// row strides, planes p = (p % n_inner, p / n_inner) with their strides.
struct ColGeom {
    long rs_in, rs_out;
    int n_inner;
    long in_inner, in_outer, out_inner, out_outer;
};

// Four-step column transform with the 32-point level on tensor cores
// (mm_tc.cu); L = 512 or 1024; forward (dir -1) reads L/2 rows, inverse
// (dir +1) writes L/2 rows.  Returns MM_OK or an error code.
int tc_cols(mm_ctx* ctx, const float2* in, float2* out, int L, int dir, int nplanes, ColGeom g, const float2* tw);
int tc_prepare(mm_ctx* ctx);

// ----- demag (mm_demag.cu)
int demag_setup(mm_ctx* ctx);                          // K1: Newell tensor -> k-space octant
int demag_apply(mm_ctx* ctx, const void* m, void* H);  // K2..K6
int demag_apply_unit(mm_ctx* ctx, const void* g, void* H);  // same with Ms = 1 (adjoint)
int demag_prepare_ff(mm_ctx* ctx);                     // float-float tables for MM_FFT_FF
int blue_prepare(mm_ctx* ctx);                         // Bluestein data of the non-power-of-two axes
// the tensor product of K4 on an unpruned R2C spectrum [3][Pz][Py][Hx] (in place)
int demag_kspace_product(mm_ctx* ctx, void* spec);
// MM_FFT_F4 (mm_f4.cu): the y forward, z product and y inverse passes fused
// over kx planes in clusters of four CTAs (FP32, ny = 512, nz = 16)
bool f4_supported(const mm_ctx* ctx);
int f4_prepare(mm_ctx* ctx);
int f4_yzy(mm_ctx* ctx, void* A);
// surrogate network: its grid, and the stream its launches go to (returns the old one)
void fno_grid(const mm_fno* f, int* nx, int* ny);
cudaStream_t fno_swap_stream(mm_fno* f, cudaStream_t s);

// ----- Newell (mm_newell.cu)
// Fills the FP64 real-space padded grid [Pz][Py][Px] of component c (0..5)
// and, when octant_out != nullptr, the octant [nz][ny][nx] of that component.
int newell_component(mm_ctx* ctx, int c, double* grid, double* octant_out, void* fgrid_scratch);

// ----- LLG and fields (mm_llg.cu)
int field_exchange(mm_ctx* ctx, const void* m, void* H);
int field_effective(mm_ctx* ctx, const void* m, const void* Hd, void* H);
int energy_launch(mm_ctx* ctx, const void* m, const void* Hd);   // adds into ctl->energy
int torque_launch(mm_ctx* ctx, const void* m, const void* Hd);   // max into ctl->torque_bits
// One RK stage: k[s] = LLG(ms_in, H_eff(ms_in)); writes next trial state or,
// at the last stage, the candidate mnext (+ error).  method MM_RK4/MM_RKF45.
int rk_stage(mm_ctx* ctx, int method, int s, const void* m_in, const void* m0, void* m_out);
int rk_controller(mm_ctx* ctx, int method);            // accept / reject, dt
int rk_commit(mm_ctx* ctx, void* m0);                  // m0 <- mnext if accepted
int check_finite_launch(mm_ctx* ctx, const void* m);
// One Barzilai-Borwein iteration after the demag field of m is in ctx->Hd:
// gradient, step length and update (no-ops once ctl->done is set).
int bb_iteration(mm_ctx* ctx, void* m, void* g, const void* g_prev, void* m_prev, bool have_prev,
                 double torque_tol, long max_iter);            // flags ctl->status
// host helpers shared with the adjoint (mm_capi.cu)
int ctl_reset_push(mm_ctx* ctx, double t, double dt, double t_max, double tol);
int ctl_pull(mm_ctx* ctx);

}  // namespace mm
