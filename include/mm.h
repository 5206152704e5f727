/*
 * mm.h - C ABI of the GB300 micromagnetic hot-path library (libmm_gb300.so).
 *
 * The library evaluates the finite-difference micromagnetic effective field
 * and integrates the Landau-Lifshitz-Gilbert equation on one NVIDIA GB300
 * (sm_103a):
 *   - demagnetisation field: the zero-padded FFT convolution of M = Ms m with
 *     the Newell tensor (paper, Implementation section, Eq. 4 and the
 *     paragraph after it; Newell's formulas are cited there, not printed);
 *   - exchange field (Eq. 2), read for the unit magnetisation m;
 *   - uniaxial anisotropy and a uniform Zeeman field (named in the
 *     Implementation section as local fields);
 *   - the LLG right-hand side (Eq. 1) for unit m, advanced with classic RK4 or
 *     Fehlberg's adaptive RKF45 (the paper's integrator, Implementation
 *     section, paragraph on ODE solvers);
 *   - energies and the maximum torque, and relax() built on RKF45.
 *
 * Conventions shared by every entry point
 *   - Units are SI: lengths in m, Ms and fields in A/m, A in J/m, Ku in J/m^3,
 *     time in s, energies in J.
 *   - Vector fields (m, H) are component-planar arrays [3][nz][ny][nx] with x
 *     fastest: component c of cell (x, y, z) sits at
 *     c*N + (z*ny + y)*nx + x, N = nx*ny*nz.  Scalar fields are [nz][ny][nx].
 *   - Element type is the context's precision: float for MM_F32, double for
 *     MM_F64.  Pointers named "device" must be device memory of the current
 *     CUDA device, 256-byte aligned (what cudaMalloc and torch give), owned by
 *     the caller, never freed or retained by the library.
 *   - Work is enqueued on the stream given at mm_init_mesh (or mm_set_stream).
 *     Calls that return host scalars (energies, torque, step errors) wait for
 *     that stream.  Calls on one context must not overlap on the host.
 *   - Mesh sizes: nx, ny any of 1..512 (powers of two take the radix-2 passes,
 *     other sizes Bluestein chirp-z passes of the next power of two >= 2P - 1,
 *     or a direct DFT when the padded length P is at most 64); nz 1 or a power
 *     of two up to 512.
 *   - Every function returns MM_OK (0) or a negative MM_ERR_* code;
 *     mm_last_error() then describes the failure.  A failed call leaves the
 *     caller's buffers in an unspecified state but the context usable, except
 *     after MM_ERR_CUDA, which reports a CUDA error of the device context.
 */
#ifndef MM_GB300_H
#define MM_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_ctx mm_ctx;

enum { MM_F32 = 0, MM_F64 = 1 };
enum { MM_RK4 = 0, MM_RKF45 = 1 };
enum { MM_DMI_INTERFACIAL = 1, MM_DMI_BULK = 2 };

enum {
    MM_OK = 0,
    MM_ERR_INVALID_ARG = -1,  /* bad size, spacing, material value or null pointer */
    MM_ERR_CUDA = -2,         /* a CUDA call failed (text in mm_last_error) */
    MM_ERR_NONFINITE = -3,    /* NaN or Inf met in m or in a step's result */
    MM_ERR_DT_UNDERFLOW = -4, /* RKF45 shrank dt below the floor (1e-20 s) */
    MM_ERR_NOT_CONVERGED = -5,/* relax() hit max_steps before torque or t_max */
    MM_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
    MM_ERR_NOMEM = -7         /* device allocation failed in mm_init_mesh */
};

/* Create a context for an nx x ny x nz mesh of dx x dy x dz cells.
 * Computes the Newell tensor on the device (double-double arithmetic),
 * transforms it and keeps its real k-space octant at the path precision;
 * allocates every scratch buffer the hot path needs (no allocation happens
 * after this call).  Material defaults: Ms = 8e5, A = 1.3e-11, alpha = 0.02,
 * Ku = 0, u = z, no external field.
 *   out        receives the context (host pointer to a host pointer)
 *   precision  MM_F32 or MM_F64
 *   stream     cudaStream_t to enqueue on (NULL = legacy default stream of
 *              the CUDA runtime's current device); the context lives on the
 *              stream's device and selects it at every call
 * Errors: INVALID_ARG (sizes, spacing <= 0, out NULL), NOMEM, CUDA. */
int mm_init_mesh(mm_ctx** out, int nx, int ny, int nz, double dx, double dy, double dz,
                 int precision, void* stream);

/* Change the stream later calls enqueue on (it must be on the context's
 * device; INVALID_ARG otherwise). */
int mm_set_stream(mm_ctx* ctx, void* stream);

/* Uniform material (Eq. 1 and 2 parameters plus anisotropy).  u_anis may be
 * NULL (then z); it is normalised.  Errors: INVALID_ARG for Ms < 0, A < 0,
 * alpha < 0, a zero u_anis. */
int mm_set_material(mm_ctx* ctx, double Ms, double A, double alpha, double Ku,
                    const double u_anis[3]);

/* Per-cell Ms and/or A ([nz][ny][nx] device arrays of the path precision);
 * NULL keeps the uniform value.  The arrays are copied; Ms = 0 marks vacuum
 * cells (no field, no motion, skipped as exchange neighbours). */
int mm_set_material_fields(mm_ctx* ctx, const void* Ms_cell, const void* A_cell);

/* Uniform external (Zeeman) field in A/m. */
int mm_set_external_field(mm_ctx* ctx, double hx, double hy, double hz);

/* Dzyaloshinskii-Moriya interaction (Eq. 3, unit m):
 *   H = 2 D / (mu0 Ms) sum_k e_k x dm/dk,
 * e_k = (e_y, -e_x, 0) for MM_DMI_INTERFACIAL, (e_x, e_y, e_z) for
 * MM_DMI_BULK; D in J/m^2 (0 switches it off).  dm/dk is the central
 * difference, and a neighbour outside the magnet (mesh edge or Ms = 0)
 * contributes nothing: the field is that of the bond energy
 * (D V / d_k) sum_bonds e_k . (m_i x m_(i+k)), which mm_energy reports as
 * E_out[4].  Enters the effective field, the LLG stages, the torque, the
 * energies and the minimiser; the adjoint entry points reject D != 0.
 * Errors: INVALID_ARG. */
int mm_set_dmi(mm_ctx* ctx, double D, int type);

/* Slonczewski spin-transfer torque (named in the paper as a local term
 * beside the effective fields; the form below is the reading taken).  In
 * Gilbert form the term gamma beta [eps m x (p x m) + eps' p x m] is added
 * to Eq. 1, beta = hbar J / (mu0 e Ms d) (A/m),
 * eps = P Lambda^2 / ((Lambda^2 + 1) + (Lambda^2 - 1) m.p); solved for dm/dt:
 *   gamma beta / (1 + alpha^2) [(eps + alpha eps') m x (p x m) - (eps' - alpha eps) m x p].
 * J current density (A/m^2; 0 switches the torque off), P polarisation,
 * Lambda >= 1, eps_prime the field-like coefficient, p[3] the fixed-layer
 * polarisation (normalised here), d the free-layer thickness in m
 * (<= 0: nz dz).  Enters the LLG stages only (not the effective field,
 * energies, torque criterion or minimiser); the adjoint entry points reject
 * it.  Set alpha with mm_set_material first: the torque's (1 + alpha^2) is
 * taken at each step from the current material.  Errors: INVALID_ARG. */
int mm_set_stt(mm_ctx* ctx, double J, double P, double Lambda, double eps_prime, const double p[3], double d);

/* H = demagnetisation field of m (Eq. 4), both device [3][nz][ny][nx].
 * FP32 contexts with ny = 256 or 512, or nx = 512, run some passes fed by
 * the copy engine (TMA) with bounded waits; a wait that gives up raises
 * TIMEOUT in the device status, which mm_llg_step, mm_relax and
 * mm_minimize_bb report (no GPU fault is involved). */
int mm_demag_field(mm_ctx* ctx, const void* m, void* H);

/* H = exchange field of m (Eq. 2), 6-point stencil, harmonic-mean A,
 * free boundary; device [3][nz][ny][nx]. */
int mm_exchange_field(mm_ctx* ctx, const void* m, void* H);

/* H = demag + exchange + anisotropy + Zeeman (at vacuum cells only the
 * demag stray field). */
int mm_effective_field(mm_ctx* ctx, const void* m, void* H);

/* One LLG step of m in place (device [3][nz][ny][nx]).
 *   method MM_RK4: fixed step *dt; *t += *dt; *err_out (nullable) = 0.
 *   method MM_RKF45: trial steps from *dt until the embedded error
 *     max_cells |m5 - m4| <= tol; on return *t is advanced by the accepted
 *     step, *dt holds the proposed next step and *err_out the accepted error.
 * m is renormalised after the step.  Errors: INVALID_ARG, NONFINITE,
 * DT_UNDERFLOW, TIMEOUT (a bounded device wait gave up), CUDA. */
int mm_llg_step(mm_ctx* ctx, void* m, double* t, double* dt, int method, double tol,
                double* err_out);

/* mm_llg_step on a host copy of the state: m_host (host [3][nz][ny][nx] of
 * the path precision; pinned memory gives the fastest copies) is copied to a
 * device buffer of the context, advanced by one step exactly as mm_llg_step
 * does, and copied back before the call returns.  The first call allocates
 * that buffer (3 N elements), kept by the context.  Errors: those of
 * mm_llg_step, INVALID_ARG for a NULL m_host, NOMEM. */
int mm_llg_step_host(mm_ctx* ctx, void* m_host, double* t, double* dt, int method, double tol,
                     double* err_out);

/* RKF45 relaxation (tol 1e-5, first dt 1e-14 s) until
 * max_cells |m x H_eff| / Ms <= torque_tol (checked every 10 trial steps,
 * sooner when fewer than 10 of the max_steps accepted steps remain) or the
 * time reaches t_max.  At most max_steps steps are accepted.  *t_out, *steps_out (nullable) receive the simulated
 * time and accepted step count.  Step-size control stays on the device.
 * Errors: NOT_CONVERGED when max_steps is reached first, NONFINITE,
 * DT_UNDERFLOW, TIMEOUT (a bounded device wait gave up), CUDA. */
int mm_relax(mm_ctx* ctx, void* m, double t_max, double torque_tol, long max_steps,
             double* t_out, long* steps_out);

/* Energy minimisation by Barzilai-Borwein steepest descent on the unit
 * sphere (the paper's minimiser, named in its Implementation section beside
 * RKF45 and called before the LLG run in its example script; the algorithm
 * is not printed there, this is the reading taken).  Per step, with
 * h = H_eff / Ms: g = m x (m x h), m <- normalise(m - tau g); tau = 1e-4 on
 * the first step, then (s.s)/(s.y) on odd and (s.y)/(y.y) on even steps
 * (s, y the changes of m and g over all cells), 1 where the quotient is not
 * positive.  Stops before a step once max |m x H_eff| / Ms <= torque_tol
 * (tested every step on the device) or after max_iter steps; *iters_out
 * (nullable) receives the steps taken.  m (device, in place) holds the last
 * state in either case.  Uses the integrator's scratch buffers.  Errors:
 * NOT_CONVERGED (max_iter reached first), NONFINITE, INVALID_ARG, TIMEOUT (a
 * bounded device wait gave up), CUDA. */
int mm_minimize_bb(mm_ctx* ctx, void* m, double torque_tol, long max_iter, long* iters_out);

/* E_out[0..4] = demag, exchange, anisotropy, Zeeman, DMI energy of m in J
 * (float64 accumulation on the device). */
int mm_energy(mm_ctx* ctx, const void* m, double E_out[5]);

/* *out = max over magnetic cells of |m x H_eff| / Ms. */
int mm_max_torque(mm_ctx* ctx, const void* m, double* out);

/* Real-space Newell tensor the context computed: host double array
 * [6][nz][ny][nx] for the non-negative offsets (i, j, k), components
 * xx, yy, zz, xy, xz, yz (negative offsets follow by parity). */
int mm_newell_tensor(mm_ctx* ctx, double* host_out);

/* Save m (device) with t and dt to a binary file; load it back into m.
 * The file records nx, ny, nz and the precision and is rejected on mismatch. */
int mm_save_state(mm_ctx* ctx, const void* m, double t, double dt, const char* path);
int mm_load_state(mm_ctx* ctx, void* m, double* t, double* dt, const char* path);

/* Free the context and everything it allocated.  NULL is a no-op. */
void mm_destroy(mm_ctx* ctx);

/* Text of the last failure on this context ("" if none).  Valid until the
 * next call on the context.  With ctx NULL: the last mm_init_mesh failure. */
const char* mm_last_error(const mm_ctx* ctx);

/* Number of kernels this context has launched since creation (all entry
 * points), for launch accounting. */
long mm_kernel_launches(const mm_ctx* ctx);

/* Kernel classes for per-kernel timing. */
enum {
    MM_K_XFWD = 0,   /* demag pass 1: x real-to-complex, pruned          */
    MM_K_YFWD = 1,   /* demag pass 2: y forward, pruned input             */
    MM_K_ZCONV = 2,  /* demag pass 3: z forward, tensor product, z inverse */
    MM_K_YINV = 3,   /* demag pass 4: y inverse, pruned output            */
    MM_K_XINV = 4,   /* demag pass 5: x complex-to-real, pruned output    */
    MM_K_STAGE = 5,  /* fused exchange + local fields + LLG + RK stage    */
    MM_K_CONTROL = 6,/* RKF45 controller and commit                       */
    MM_K_REDUCE = 7, /* energies, torque, finiteness check, field kernels */
    MM_K_COUNT = 8
};

/* Turn per-kernel timing on (1) or off (0).  When on, every launch of the
 * context is bracketed by CUDA events recorded on the context's stream.
 * Turning it on clears the accumulated times. */
int mm_enable_kernel_timing(mm_ctx* ctx, int enable);

/* The same for a subset of kernel classes (no paper counterpart):
 * bit k of `classes` (k < MM_K_COUNT) brackets the launches of class k with
 * events; launches of every class are counted while any bit is set; 0 turns
 * timing off.  Each event pair costs device time, so timing one class keeps
 * the measured stretch closer to an uninstrumented run.  Clears the
 * accumulated times.  Errors: INVALID_ARG (bits above MM_K_COUNT). */
int mm_enable_kernel_timing_mask(mm_ctx* ctx, unsigned classes);

/* Waits for the stream, then reports the summed device time (ms, 0 for a
 * class outside the timing mask) and the launch count of kernel class
 * `kernel` since timing was enabled. */
int mm_kernel_time(mm_ctx* ctx, int kernel, double* total_ms, long* launches);

/* After any call that waited for the stream (llg_step, relax, energy,
 * torque): accepted steps, rejected RKF45 trials, time and next dt of the
 * last integration call.  Any pointer may be NULL. */
int mm_step_stats(const mm_ctx* ctx, long* accepted, long* rejected, double* t, double* dt);

/* Kinds of mm_alu_peak. */
enum { MM_ROOF_FP64 = 0, MM_ROOF_FP32 = 1, MM_ROOF_FP32X2 = 2 };

/* Measured arithmetic roof of this GPU for the ALU-bound paths: *flops_per_s
 * receives the FMA throughput of a kernel that keeps 8 independent FMA
 * chains per thread on 8 blocks per SM (best of three timed launches after
 * one warm-up), counted as 2 flops per FMA: fma.rn.f64 (MM_ROOF_FP64, the
 * roof of the native FP64 passes), fma.rn.f32 (MM_ROOF_FP32) or
 * fma.rn.f32x2 on lane pairs (MM_ROOF_FP32X2; the roof of the float-float
 * passes).  stream as in mm_init_mesh; the caller's current device is
 * restored.  Instrumentation only: allocates and frees a small buffer and
 * two events per call.  Errors: INVALID_ARG, CUDA. */
int mm_alu_peak(int kind, double* flops_per_s, void* stream);

/* The tensor product of the demag convolution (Eq. 4 in k-space,
 * H^ = -N^ M^) applied in place to an UNPRUNED real-to-complex spectrum of
 * the whole padded grid: device complex array [3][Pz][Py][Px/2+1] of the
 * path precision (x fastest; Px, Py, Pz = 2n per axis, 1 where n = 1), the
 * layout a library R2C transform over the three padded axes produces.  It
 * uses the context's Newell octant with the components' parities.  An
 * unnormalised inverse C2R transform of the result, divided by Px Py Pz and
 * cut to the mesh, is the demagnetisation field.  This exists so that a
 * library FFT (cuFFT) can be timed against the library's pruned passes on
 * the same kernel; the library's own path never calls it.  Errors:
 * INVALID_ARG, CUDA. */
int mm_kspace_product(mm_ctx* ctx, void* spectrum);

/* ---- Adjoints (gradients with respect to m and the per-cell Ms) ------------
 * The paper names automatic differentiation for inverse problems as a
 * property of its PyTorch base (Introduction); these are hand-written
 * vector-Jacobian products of Eq. 1, 2 and 4 for that use.  Cotangents and
 * gradients are device arrays of the path precision: vector fields
 * [3][nz][ny][nx], gMs [nz][ny][nx] (accumulated: gMs += ..., zero it
 * first).  The per-cell Ms used is the context's (mm_set_material_fields),
 * else the uniform value.  The first adjoint call allocates a workspace of
 * 14 vector fields kept by the context. */

/* gm = (dH_demag/dm)^T g = Ms (-N * g); gMs += m . (-N * g) (gMs nullable).
 * The Newell operator is symmetric and even, hence self-adjoint. */
int mm_demag_vjp(mm_ctx* ctx, const void* g, const void* m, void* gm, void* gMs);

/* gm = (dH_ex/dm)^T g = E(g / Ms), E the symmetric exchange stencil;
 * gMs += -g . H_ex(m) / Ms (gMs nullable). */
int mm_exchange_vjp(mm_ctx* ctx, const void* g, const void* m, void* gm, void* gMs);

/* One classic RK4 step m1 = u/|u|, u = m0 + dt sum b_s k_s (Eq. 1 with the
 * full effective field): lam holds dL/dm1 on entry and dL/dm0 on return;
 * gMs += (dm1/dMs)^T lam.  The stage states are recomputed from m0. */
int mm_rk4_step_vjp(mm_ctx* ctx, const void* m0, double dt, void* lam, void* gMs);

/* nsteps fixed RK4 steps of m in place without host synchronisation
 * between steps; waits for the stream at the end. */
int mm_rk4_trajectory(mm_ctx* ctx, void* m, double dt, long nsteps);

/* Reverse pass of mm_rk4_trajectory from m0: lam = dL/dm_N on entry,
 * dL/dm_0 on return; gMs += dL/dMs.  Checkpoints the state every
 * checkpoint_every steps (<= 0: ceil(sqrt(nsteps))) and replays each
 * segment before pulling back through it, so memory is about
 * (nsteps / K + K) states.  While a segment is replayed, each step's stage
 * states, demag fields and slopes (10 K states) are recorded when they fit
 * in 16 GiB, so the step VJPs need not recompute them; otherwise each step
 * VJP recomputes its stages.  All of it is allocated for the call and freed
 * before it returns. */
int mm_rk4_trajectory_vjp(mm_ctx* ctx, const void* m0, double dt, long nsteps, void* lam, void* gMs,
                          long checkpoint_every);

/* ---- Tensor-core split-precision DFT stage ----------------------------------
 * The paper's FFTs run in FP64/FP32 through cuFFT; this is the precision
 * variant of its radix stages: a 32-point DFT as a real GEMM on the
 * 5th-generation tensor cores, FP32 operands split into hi + lo parts of the
 * tensor-core type and multiplied as hi.hi + hi.lo + lo.hi with FP32
 * accumulation (about 21 significant bits for TF32, 16 for BF16). */
enum { MM_TC_TF32 = 1, MM_TC_BF16 = 2, MM_FFT_FF = 3, MM_FFT_F4 = 4 };

/* out[l][k] = sum_n in[l][n] exp(direction 2 pi i n k / 32) for nlines
 * lines of 32 complex FP32 values (interleaved re, im; device arrays,
 * in != out).  direction -1 or +1.  Waits for the stream.  Errors:
 * INVALID_ARG, CUDA, TIMEOUT (a bounded tensor-core wait gave up; read with
 * mm_last_error(NULL)). */
int mm_dft32_tc(const void* in, void* out, long nlines, int mode, int direction, void* stream);

/* FFT arithmetic of a context's demag passes (Implementation section,
 * Eq. 4: the convolution itself is unchanged, only the arithmetic that
 * evaluates its transforms).  0 = the context's own precision (default).
 * MM_F32 context: MM_TC_TF32 or MM_TC_BF16 = the y passes of length 512 or
 * 1024 run their 32-point level on tensor cores with split operands (the
 * other passes stay FP32): TF32 in hi + lo parts (about 21 bits), BF16 in
 * hi + mid + lo parts with the six products down to 2^-23 (about 24 bits,
 * within the FP32 tolerance).
 * MM_F64 context: MM_FFT_FF = all five passes in float-float arithmetic
 * (pairs of FP32 values, about 48 significant bits, on the FP32 pipes), and,
 * for uniform Ms and A without DMI or STT, the LLG stage kernel as well
 * (its renormalisation finished in float64); m, Ms, H, the stage slopes and
 * everything else stay float64 arrays; the padded sizes Px, Py, Pz must be
 * powers of two.  Setting it allocates float-float
 * copies of the Newell octant and twiddle tables (6 (Pz/2+1)(Py/2+1) Hs x 8
 * bytes plus the tables), kept until mm_destroy.
 * MM_F32 context with ny = 512 and nz = 16: MM_FFT_F4 = the y forward pass,
 * the z transform with the tensor product and the y inverse pass fused into
 * one pass over kx planes, each held on chip by a cluster of four CTAs (the
 * 3-pass thin-film variant: the spectrum crosses HBM once between the x
 * passes instead of three times); setting it allocates a copy of the octant
 * laid out per kx plane (Hx x 4 x 6 x (Pz/2+1) x 256 floats) and a twiddle
 * table, kept until mm_destroy.
 * Errors: INVALID_ARG (unknown mode, mode not valid for the context's
 * precision or mesh), NOMEM/CUDA (allocation or setup). */
int mm_set_fft_mode(mm_ctx* ctx, int mode);

/* MM_OK, or MM_ERR_TIMEOUT if a tensor-core wait of this device gave up
 * since the last check (waits for the stream). */
int mm_tc_status(mm_ctx* ctx);

/* Self-test of the library's bounded device waits (no paper counterpart):
 * one block polls an mbarrier that nothing completes, `limit` times
 * (1 .. 2^20), the same way the tensor-core kernels wait for their MMAs,
 * gives up, and raises TIMEOUT in the device status.  The call reads the
 * status, clears it again and returns MM_ERR_TIMEOUT when the wait gave up
 * as designed (MM_OK would mean it did not); no GPU fault is involved and
 * the library stays usable.  Uses one cudaMalloc of 4 bytes.  stream:
 * cudaStream_t or NULL.  Errors: INVALID_ARG, CUDA. */
int mm_tc_wait_selftest(long limit, void* stream);

/* ---- Fourier-neural-operator surrogate of the demag field ------------------
 * Not in the paper: a learned stand-in for Eq. 4 on 2-D films (nz = 1), used
 * inside relax() with the exact field recomputed every k steps.  Network:
 * lift 3 -> width (1x1), `layers` Fourier layers a = W v + b +
 * IDFT(R . DFT v) on the retained modes kx < modes, ky < modes or
 * ky >= ny - modes, GELU between layers, projection width -> 3 (1x1).
 * Maps m [B][3][ny][nx] to h = H_demag / Ms [B][3][ny][nx] (FP32 device
 * arrays).  Activations are stored as BF16 (store_bf16 = 1) or FP32, every
 * contraction accumulates in FP32; parameters are FP32.  Errors go to
 * mm_last_error(NULL). */
typedef struct mm_fno mm_fno;
int mm_fno_create(mm_fno** out, int nx, int ny, int width, int modes, int layers, int store_bf16,
                  int max_batch, unsigned long long seed, void* stream);
void mm_fno_destroy(mm_fno* f);
long mm_fno_num_params(const mm_fno* f);
/* h = FNO(m) for `batch` samples; keeps the activations for mm_fno_backward. */
int mm_fno_forward(mm_fno* f, const void* m, void* h, int batch);
/* Accumulates dL/dparams (gradients += ...) for cotangent dh of the last
 * forward call on the same m. */
int mm_fno_backward(mm_fno* f, const void* m, const void* dh, int batch);
int mm_fno_zero_grad(mm_fno* f);
int mm_fno_adam_step(mm_fno* f, double lr, double beta1, double beta2, double eps, long step);
/* Mean over samples of |h - target|^2 / |target|^2 (*loss_out, nullable,
 * waits for the stream); dh (nullable) receives its gradient. */
int mm_fno_loss(mm_fno* f, const void* h, const void* target, void* dh, int batch, double* loss_out);
/* Host copies: read parameters / gradients (nullable), or set parameters
 * from host_set (nullable); mm_fno_num_params floats each. */
int mm_fno_params(mm_fno* f, float* host_params, float* host_grads, const float* host_set);
/* Output multiplier (1 for training; Ms when the output stands in for H). */
int mm_fno_set_output_scale(mm_fno* f, double scale);

/* relax() with the surrogate: every k_exact accepted-step window starts
 * with the exact demag field of the current state and the maximum torque of
 * the exact effective field; the call stops like mm_relax on that torque,
 * so the relaxed state meets the same criterion as mm_relax's.  A window
 * whose start torque is at or below torque_exact (the final approach) runs
 * on the exact field.  Above it, the surrogate's field of the same state is
 * checked against the exact one: with a relative L2 residual of at most
 * `bound` the window's RKF45 stage demag fields come from the surrogate,
 * otherwise from the exact FFT convolution (a fallback), and the next check
 * waits 1, 2, 4, ... (at most 64) windows while consecutive checks fail.
 * MM_F32 context, nz = 1, uniform Ms, surrogate of the same grid (its
 * launches go to the context's stream for the call).  stats (nullable, 3
 * longs): exact demag evaluations, surrogate evaluations, failed checks.
 * One call at a time per surrogate: the call sets the surrogate's stream
 * and output scale for its duration. */
int mm_relax_surrogate(mm_ctx* ctx, mm_fno* f, void* m, double t_max, double torque_tol, long max_steps,
                       int k_exact, double bound, double torque_exact, double* t_out, long* steps_out, long* stats);

/* Energies without a context and without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory themselves or through this library (for
 * example code that runs inside a memory pool or arena it does not own, or a
 * plugin that is handed only its host application's buffers), and so cannot
 * create a context.  It computes what mm_energy computes (E_out[0..3] =
 * demag, exchange, anisotropy, Zeeman energy in J) for a uniform material
 * without DMI,
 * taking the demagnetisation field H_demag from the caller (for instance
 * from mm_demag_field) instead of evaluating it.
 *   m, H_demag  device arrays [3][nz][ny][nx] of the given precision
 *   u_anis      anisotropy axis (NULL = z, normalised); h_ext Zeeman field in
 *               A/m (NULL = none); E_out host array of 4 doubles
 *   stream      cudaStream_t (NULL = legacy default stream of the current
 *               device); the call waits for it before returning.  A stream
 *               of another device is served on that device, which is made
 *               current for the call; the caller's current device is
 *               restored before the call returns, on success and on error
 * Scratch: block partial sums live in one fixed array of 1 MiB in the
 * library's device memory, which every GPU that loads the library keeps
 * until the process exits.  Meshes above 8,388,608 cells are rejected with
 * INVALID_ARG.  The call uses no cudaMalloc or cudaFree.  The first call on
 * each device looks up the array's device address; make that first call
 * before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU race and must be serialised by the caller.
 * Errors (read with mm_last_error(NULL)): INVALID_ARG, CUDA. */
int mm_energy_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, int precision,
                      double Ms, double A, double Ku, const double u_anis[3], const double h_ext[3],
                      const void* m, const void* H_demag, double E_out[4], void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MM_GB300_H */
