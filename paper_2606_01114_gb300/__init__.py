"""Python binding of libmm_gb300.so, the GB300 micromagnetic hot-path library.

Argument marshalling only: every function forwards to the C entry point of
the same name in ``include/mm.h`` and raises ``MMError`` on a non-zero return
code.  Device arrays are torch CUDA tensors (or any object with ``data_ptr``,
``is_cuda``, ``dtype``, ``shape`` and ``is_contiguous``), vector fields shaped
(3, nz, ny, nx), scalars (nz, ny, nx), dtype float32 for MM_F32 contexts and
float64 for MM_F64.  All compute happens in the library's CUDA kernels; if
the library is not built, loading fails loudly.

Conversions from the paper's (nx, ny, nz, 3) layout: ``from_paper_layout`` /
``to_paper_layout``.
"""

import ctypes
import os

import numpy as np

MM_F32, MM_F64 = 0, 1
MM_RK4, MM_RKF45 = 0, 1
MM_DMI_INTERFACIAL, MM_DMI_BULK = 1, 2
MM_OK = 0
MM_ERR_INVALID_ARG = -1
MM_ERR_CUDA = -2
MM_ERR_NONFINITE = -3
MM_ERR_DT_UNDERFLOW = -4
MM_ERR_NOT_CONVERGED = -5
MM_ERR_TIMEOUT = -6
MM_ERR_NOMEM = -7
MM_TC_TF32, MM_TC_BF16, MM_FFT_FF, MM_FFT_F4 = 1, 2, 3, 4
MM_ROOF_FP64, MM_ROOF_FP32, MM_ROOF_FP32X2 = 0, 1, 2
# kernel classes for mm_kernel_time
MM_K_XFWD, MM_K_YFWD, MM_K_ZCONV, MM_K_YINV, MM_K_XINV, MM_K_STAGE, MM_K_CONTROL, MM_K_REDUCE = range(8)
MM_K_COUNT = 8
KERNEL_NAMES = ("xfwd", "yfwd", "zconv", "yinv", "xinv", "stage", "control", "reduce")

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmm_gb300.so")
_lib = None


class MMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2606_01114_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
    DP = ctypes.POINTER(ctypes.c_double)
    LP = ctypes.POINTER(ctypes.c_long)
    sig = {
        "mm_init_mesh": (I, [ctypes.POINTER(P), I, I, I, D, D, D, I, P]),
        "mm_set_stream": (I, [P, P]),
        "mm_set_material": (I, [P, D, D, D, D, DP]),
        "mm_set_material_fields": (I, [P, P, P]),
        "mm_set_external_field": (I, [P, D, D, D]),
        "mm_demag_field": (I, [P, P, P]),
        "mm_exchange_field": (I, [P, P, P]),
        "mm_effective_field": (I, [P, P, P]),
        "mm_llg_step": (I, [P, P, DP, DP, I, D, DP]),
        "mm_relax": (I, [P, P, D, D, L, DP, LP]),
        "mm_energy": (I, [P, P, DP]),
        "mm_max_torque": (I, [P, P, DP]),
        "mm_newell_tensor": (I, [P, DP]),
        "mm_save_state": (I, [P, P, D, D, ctypes.c_char_p]),
        "mm_load_state": (I, [P, P, DP, DP, ctypes.c_char_p]),
        "mm_destroy": (None, [P]),
        "mm_last_error": (ctypes.c_char_p, [P]),
        "mm_kernel_launches": (L, [P]),
        "mm_enable_kernel_timing": (I, [P, I]),
        "mm_enable_kernel_timing_mask": (I, [P, ctypes.c_uint]),
        "mm_kernel_time": (I, [P, I, DP, LP]),
        "mm_step_stats": (I, [P, LP, LP, DP, DP]),
        "mm_energy_noalloc": (I, [I, I, I, D, D, D, I, D, D, D, DP, DP, P, P, DP, P]),
        "mm_demag_vjp": (I, [P, P, P, P, P]),
        "mm_exchange_vjp": (I, [P, P, P, P, P]),
        "mm_rk4_step_vjp": (I, [P, P, D, P, P]),
        "mm_rk4_trajectory": (I, [P, P, D, L]),
        "mm_rk4_trajectory_vjp": (I, [P, P, D, L, P, P, L]),
        "mm_dft32_tc": (I, [P, P, L, I, I, P]),
        "mm_set_fft_mode": (I, [P, I]),
        "mm_tc_status": (I, [P]),
        "mm_fno_create": (I, [ctypes.POINTER(P), I, I, I, I, I, I, I, ctypes.c_ulonglong, P]),
        "mm_fno_destroy": (None, [P]),
        "mm_fno_num_params": (L, [P]),
        "mm_fno_forward": (I, [P, P, P, I]),
        "mm_fno_backward": (I, [P, P, P, I]),
        "mm_fno_zero_grad": (I, [P]),
        "mm_fno_adam_step": (I, [P, D, D, D, D, L]),
        "mm_fno_loss": (I, [P, P, P, P, I, DP]),
        "mm_fno_params": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                              ctypes.POINTER(ctypes.c_float)]),
        "mm_fno_set_output_scale": (I, [P, D]),
        "mm_set_dmi": (I, [P, D, I]),
        "mm_set_stt": (I, [P, D, D, D, D, P, D]),
        "mm_tc_wait_selftest": (I, [L, P]),
        "mm_minimize_bb": (I, [P, P, D, L, LP]),
        "mm_relax_surrogate": (I, [P, P, P, D, D, L, I, D, D, DP, LP, LP]),
        "mm_llg_step_host": (I, [P, P, DP, DP, I, D, DP]),
        "mm_alu_peak": (I, [I, DP, P]),
        "mm_kspace_product": (I, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Context:
    """Handle returned by ``mm_init_mesh``: the C context plus its shape."""

    def __init__(self, handle, n, d, precision):
        self.handle = handle
        self.n = tuple(n)
        self.d = tuple(d)
        self.precision = precision

    @property
    def shape3(self):
        nx, ny, nz = self.n
        return (3, nz, ny, nx)

    @property
    def shape1(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mm_destroy(self.handle)
            self.handle = None


def _check(ctx, rc):
    if rc != MM_OK:
        h = ctx.handle if isinstance(ctx, Context) else None
        raise MMError(rc, _load().mm_last_error(h).decode())


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(ctx, t, shape, name):
    if t is None:
        return None
    want = "float64" if ctx.precision == MM_F64 else "float32"
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype).split(".")[-1] != want:
        raise ValueError(f"{name} must be {want} for this context, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def mm_init_mesh(nx, ny, nz, dx, dy, dz, precision=MM_F32, stream=None):
    lib = _load()
    h = ctypes.c_void_p()
    rc = lib.mm_init_mesh(ctypes.byref(h), int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                          int(precision), _stream_ptr(stream))
    if rc != MM_OK:
        raise MMError(rc, lib.mm_last_error(None).decode())
    return Context(h, (nx, ny, nz), (dx, dy, dz), precision)


def mm_set_stream(ctx, stream):
    _check(ctx, _load().mm_set_stream(ctx.handle, _stream_ptr(stream)))


def mm_set_material(ctx, Ms, A, alpha, Ku=0.0, u=None):
    uu = None if u is None else (ctypes.c_double * 3)(*[float(v) for v in u])
    _check(ctx, _load().mm_set_material(ctx.handle, float(Ms), float(A), float(alpha), float(Ku), uu))


def mm_set_material_fields(ctx, Ms_cell=None, A_cell=None):
    _check(ctx, _load().mm_set_material_fields(ctx.handle, _dev(ctx, Ms_cell, ctx.shape1, "Ms_cell"),
                                               _dev(ctx, A_cell, ctx.shape1, "A_cell")))


def mm_set_external_field(ctx, hx, hy, hz):
    _check(ctx, _load().mm_set_external_field(ctx.handle, float(hx), float(hy), float(hz)))


def mm_set_dmi(ctx, D, kind=MM_DMI_INTERFACIAL):
    _check(ctx, _load().mm_set_dmi(ctx.handle, float(D), int(kind)))


def mm_set_stt(ctx, J, P, Lambda, eps_prime, p, d=0.0):
    pp = (ctypes.c_double * 3)(*[float(v) for v in p])
    _check(ctx, _load().mm_set_stt(ctx.handle, float(J), float(P), float(Lambda), float(eps_prime), pp, float(d)))


def mm_demag_field(ctx, m, H):
    _check(ctx, _load().mm_demag_field(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), _dev(ctx, H, ctx.shape3, "H")))


def mm_exchange_field(ctx, m, H):
    _check(ctx, _load().mm_exchange_field(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), _dev(ctx, H, ctx.shape3, "H")))


def mm_effective_field(ctx, m, H):
    _check(ctx, _load().mm_effective_field(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), _dev(ctx, H, ctx.shape3, "H")))


def mm_llg_step(ctx, m, t, dt, method=MM_RK4, tol=1e-5):
    """Returns (t, dt, err) after one accepted step of m in place."""
    tt, dd, ee = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_double(0.0)
    _check(ctx, _load().mm_llg_step(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), ctypes.byref(tt), ctypes.byref(dd),
                                     int(method), float(tol), ctypes.byref(ee)))
    return tt.value, dd.value, ee.value


def mm_llg_step_host(ctx, m_host, t, dt, method=MM_RK4, tol=1e-5):
    """mm_llg_step on a host array (numpy or CPU tensor, C-contiguous, shape
    (3, nz, ny, nx), the context's dtype), updated in place.  Returns
    (t, dt, err)."""
    want = np.float64 if ctx.precision == MM_F64 else np.float32
    if hasattr(m_host, "data_ptr"):
        if getattr(m_host, "is_cuda", False) or str(m_host.dtype).split(".")[-1] != np.dtype(want).name:
            raise ValueError(f"m_host must be a CPU {np.dtype(want).name} tensor")
        if tuple(m_host.shape) != ctx.shape3 or not m_host.is_contiguous():
            raise ValueError(f"m_host must be contiguous with shape {ctx.shape3}")
        ptr = m_host.data_ptr()
    else:
        if m_host.dtype != want or m_host.shape != ctx.shape3 or not m_host.flags.c_contiguous:
            raise ValueError(f"m_host must be a C-contiguous {np.dtype(want).name} array of shape {ctx.shape3}")
        ptr = m_host.ctypes.data
    tt, dd, ee = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_double(0.0)
    _check(ctx, _load().mm_llg_step_host(ctx.handle, ctypes.c_void_p(ptr), ctypes.byref(tt), ctypes.byref(dd),
                                          int(method), float(tol), ctypes.byref(ee)))
    return tt.value, dd.value, ee.value


def mm_relax(ctx, m, t_max, torque_tol=1e-4, max_steps=1000000):
    """Returns (t, accepted_steps)."""
    tt, ss = ctypes.c_double(0.0), ctypes.c_long(0)
    _check(ctx, _load().mm_relax(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), float(t_max), float(torque_tol),
                                 int(max_steps), ctypes.byref(tt), ctypes.byref(ss)))
    return tt.value, ss.value


def mm_minimize_bb(ctx, m, torque_tol=1e-4, max_iter=100000):
    """Barzilai-Borwein energy minimisation of m in place; returns the steps taken."""
    it = ctypes.c_long(0)
    _check(ctx, _load().mm_minimize_bb(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), float(torque_tol), int(max_iter),
                                       ctypes.byref(it)))
    return it.value


def mm_energy(ctx, m):
    E = (ctypes.c_double * 5)()
    _check(ctx, _load().mm_energy(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), E))
    return np.array(E[:])


def mm_max_torque(ctx, m):
    out = ctypes.c_double(0.0)
    _check(ctx, _load().mm_max_torque(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), ctypes.byref(out)))
    return out.value


def mm_newell_tensor(ctx):
    nx, ny, nz = ctx.n
    out = np.empty((6, nz, ny, nx), dtype=np.float64)
    _check(ctx, _load().mm_newell_tensor(ctx.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def mm_save_state(ctx, m, t, dt, path):
    _check(ctx, _load().mm_save_state(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), float(t), float(dt),
                                      os.fsencode(path)))


def mm_load_state(ctx, m, path):
    tt, dd = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(ctx, _load().mm_load_state(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), ctypes.byref(tt), ctypes.byref(dd),
                                      os.fsencode(path)))
    return tt.value, dd.value


def mm_destroy(ctx):
    if ctx.handle:
        _load().mm_destroy(ctx.handle)
        ctx.handle = None


def mm_last_error(ctx=None):
    return _load().mm_last_error(ctx.handle if ctx is not None else None).decode()


def mm_kernel_launches(ctx):
    return int(_load().mm_kernel_launches(ctx.handle))


def mm_enable_kernel_timing(ctx, enable=True):
    _check(ctx, _load().mm_enable_kernel_timing(ctx.handle, 1 if enable else 0))


def mm_enable_kernel_timing_mask(ctx, classes):
    """Time only the kernel classes whose bits are set in `classes` (every
    class's launches are still counted); 0 turns timing off."""
    _check(ctx, _load().mm_enable_kernel_timing_mask(ctx.handle, int(classes)))


def mm_kernel_time(ctx, kernel):
    """Returns (total_ms, launches) of kernel class ``kernel`` since timing was enabled."""
    ms, n = ctypes.c_double(0.0), ctypes.c_long(0)
    _check(ctx, _load().mm_kernel_time(ctx.handle, int(kernel), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def mm_step_stats(ctx):
    """Returns (accepted, rejected, t, dt) of the last integration call."""
    a, r = ctypes.c_long(0), ctypes.c_long(0)
    t, dt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(ctx, _load().mm_step_stats(ctx.handle, ctypes.byref(a), ctypes.byref(r), ctypes.byref(t), ctypes.byref(dt)))
    return a.value, r.value, t.value, dt.value


def mm_demag_vjp(ctx, g, m, gm, gMs=None):
    _check(ctx, _load().mm_demag_vjp(ctx.handle, _dev(ctx, g, ctx.shape3, "g"), _dev(ctx, m, ctx.shape3, "m"),
                                      _dev(ctx, gm, ctx.shape3, "gm"), _dev(ctx, gMs, ctx.shape1, "gMs")))


def mm_exchange_vjp(ctx, g, m, gm, gMs=None):
    _check(ctx, _load().mm_exchange_vjp(ctx.handle, _dev(ctx, g, ctx.shape3, "g"), _dev(ctx, m, ctx.shape3, "m"),
                                         _dev(ctx, gm, ctx.shape3, "gm"), _dev(ctx, gMs, ctx.shape1, "gMs")))


def mm_rk4_step_vjp(ctx, m0, dt, lam, gMs):
    _check(ctx, _load().mm_rk4_step_vjp(ctx.handle, _dev(ctx, m0, ctx.shape3, "m0"), float(dt),
                                         _dev(ctx, lam, ctx.shape3, "lam"), _dev(ctx, gMs, ctx.shape1, "gMs")))


def mm_rk4_trajectory(ctx, m, dt, nsteps):
    _check(ctx, _load().mm_rk4_trajectory(ctx.handle, _dev(ctx, m, ctx.shape3, "m"), float(dt), int(nsteps)))


def mm_rk4_trajectory_vjp(ctx, m0, dt, nsteps, lam, gMs, checkpoint_every=0):
    _check(ctx, _load().mm_rk4_trajectory_vjp(ctx.handle, _dev(ctx, m0, ctx.shape3, "m0"), float(dt), int(nsteps),
                                               _dev(ctx, lam, ctx.shape3, "lam"), _dev(ctx, gMs, ctx.shape1, "gMs"),
                                               int(checkpoint_every)))


def mm_set_fft_mode(ctx, mode):
    """0 = the context's own precision; MM_TC_TF32 / MM_TC_BF16 = tensor-core
    y passes (MM_F32 context); MM_FFT_FF = float-float demag passes (MM_F64
    context, power-of-two padded sizes)."""
    _check(ctx, _load().mm_set_fft_mode(ctx.handle, int(mode)))


def mm_tc_status(ctx):
    _check(ctx, _load().mm_tc_status(ctx.handle))


def mm_dft32_tc(inp, out, mode=MM_TC_TF32, direction=-1, stream=None):
    """Batched 32-point complex DFT on tensor cores (split hi + lo operands).
    inp, out: complex64 CUDA tensors of shape (nlines, 32)."""
    for name, t in (("inp", inp), ("out", out)):
        if not getattr(t, "is_cuda", False) or str(t.dtype).split(".")[-1] != "complex64" or t.shape[-1] != 32:
            raise ValueError(f"{name} must be a complex64 CUDA tensor with 32 values per line")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    lib = _load()
    rc = lib.mm_dft32_tc(ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(inp.numel() // 32),
                         int(mode), int(direction), _stream_ptr(stream))
    if rc != MM_OK:
        raise MMError(rc, lib.mm_last_error(None).decode())


def mm_tc_wait_selftest(limit=1000, stream=None):
    """Runs the bounded-wait self-test; returns its code (MM_ERR_TIMEOUT when
    the wait gave up as designed) without raising."""
    return int(_load().mm_tc_wait_selftest(int(limit), _stream_ptr(stream)))


def mm_energy_noalloc(n, d, precision, Ms, A, Ku, u, h_ext, m, H_demag, stream=None):
    """Energies (demag, exchange, anisotropy, Zeeman) without a context and
    without any device allocation; H_demag is supplied by the caller.  For
    callers that cannot allocate device memory (see include/mm.h)."""
    nx, ny, nz = (int(v) for v in n)
    want = "float64" if precision == MM_F64 else "float32"
    for name, t in (("m", m), ("H_demag", H_demag)):
        if not getattr(t, "is_cuda", False) or str(t.dtype).split(".")[-1] != want:
            raise ValueError(f"{name} must be a {want} CUDA tensor")
        if tuple(t.shape) != (3, nz, ny, nx) or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {(3, nz, ny, nx)}")
    uu = None if u is None else (ctypes.c_double * 3)(*[float(v) for v in u])
    hh = None if h_ext is None else (ctypes.c_double * 3)(*[float(v) for v in h_ext])
    E = (ctypes.c_double * 4)()
    lib = _load()
    rc = lib.mm_energy_noalloc(nx, ny, nz, float(d[0]), float(d[1]), float(d[2]), int(precision), float(Ms),
                               float(A), float(Ku), uu, hh, ctypes.c_void_p(m.data_ptr()),
                               ctypes.c_void_p(H_demag.data_ptr()), E, _stream_ptr(stream))
    if rc != MM_OK:
        raise MMError(rc, lib.mm_last_error(None).decode())
    return np.array(E[:])


def mm_alu_peak(kind=MM_ROOF_FP64, stream=None):
    """Measured FMA throughput in flop/s (2 flops per FMA) of this GPU for
    MM_ROOF_FP64, MM_ROOF_FP32 or MM_ROOF_FP32X2."""
    out = ctypes.c_double(0.0)
    lib = _load()
    rc = lib.mm_alu_peak(int(kind), ctypes.byref(out), _stream_ptr(stream))
    if rc != MM_OK:
        raise MMError(rc, lib.mm_last_error(None).decode())
    return out.value


def mm_kspace_product(ctx, spectrum):
    """In-place -N^ M^ on an unpruned R2C spectrum (complex tensor of shape
    (3, Pz, Py, Px // 2 + 1) on the context's device, complex64 for MM_F32,
    complex128 for MM_F64)."""
    nx, ny, nz = ctx.n
    shape = (3, 2 * nz if nz > 1 else 1, 2 * ny if ny > 1 else 1, nx + 1 if nx > 1 else 1)
    want = "complex128" if ctx.precision == MM_F64 else "complex64"
    if not getattr(spectrum, "is_cuda", False) or str(spectrum.dtype).split(".")[-1] != want:
        raise ValueError(f"spectrum must be a {want} CUDA tensor")
    if tuple(spectrum.shape) != shape or not spectrum.is_contiguous():
        raise ValueError(f"spectrum must be contiguous with shape {shape}")
    _check(ctx, _load().mm_kspace_product(ctx.handle, ctypes.c_void_p(spectrum.data_ptr())))


class FNO:
    """Handle of an ``mm_fno`` (created by ``mm_fno_create``)."""

    def __init__(self, handle, nx, ny, max_batch):
        self.handle, self.nx, self.ny, self.max_batch = handle, nx, ny, max_batch

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mm_fno_destroy(self.handle)
            self.handle = None


def _fcheck(rc):
    if rc != MM_OK:
        raise MMError(rc, _load().mm_last_error(None).decode())


def _f32(t, shape, name):
    if not getattr(t, "is_cuda", False) or str(t.dtype).split(".")[-1] != "float32" or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape[-3:]) != tuple(shape):
        raise ValueError(f"{name} must end in shape {shape}")
    return ctypes.c_void_p(t.data_ptr())


def mm_fno_create(nx, ny, width=32, modes=16, layers=4, store_bf16=True, max_batch=16, seed=0, stream=None):
    h = ctypes.c_void_p()
    _fcheck(_load().mm_fno_create(ctypes.byref(h), int(nx), int(ny), int(width), int(modes), int(layers),
                                  1 if store_bf16 else 0, int(max_batch), int(seed), _stream_ptr(stream)))
    return FNO(h, nx, ny, max_batch)


def mm_fno_destroy(f):
    if f.handle:
        _load().mm_fno_destroy(f.handle)
        f.handle = None


def mm_fno_num_params(f):
    return int(_load().mm_fno_num_params(f.handle))


def mm_fno_forward(f, m, h):
    _fcheck(_load().mm_fno_forward(f.handle, _f32(m, (3, f.ny, f.nx), "m"), _f32(h, (3, f.ny, f.nx), "h"),
                                   int(m.numel() // (3 * f.nx * f.ny))))


def mm_fno_backward(f, m, dh):
    _fcheck(_load().mm_fno_backward(f.handle, _f32(m, (3, f.ny, f.nx), "m"), _f32(dh, (3, f.ny, f.nx), "dh"),
                                    int(m.numel() // (3 * f.nx * f.ny))))


def mm_fno_zero_grad(f):
    _fcheck(_load().mm_fno_zero_grad(f.handle))


def mm_fno_adam_step(f, lr, beta1=0.9, beta2=0.999, eps=1e-8, step=1):
    _fcheck(_load().mm_fno_adam_step(f.handle, float(lr), float(beta1), float(beta2), float(eps), int(step)))


def mm_fno_loss(f, h, target, dh=None):
    out = ctypes.c_double(0.0)
    _fcheck(_load().mm_fno_loss(f.handle, _f32(h, (3, f.ny, f.nx), "h"), _f32(target, (3, f.ny, f.nx), "target"),
                                None if dh is None else _f32(dh, (3, f.ny, f.nx), "dh"),
                                int(h.numel() // (3 * f.nx * f.ny)), ctypes.byref(out)))
    return out.value


def mm_fno_params(f, set_params=None):
    """Returns (params, grads) as float32 numpy arrays; sets parameters first if given."""
    n = mm_fno_num_params(f)
    p = np.empty(n, dtype=np.float32)
    g = np.empty(n, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    s = None if set_params is None else np.ascontiguousarray(set_params, dtype=np.float32)
    _fcheck(_load().mm_fno_params(f.handle, p.ctypes.data_as(fp), g.ctypes.data_as(fp),
                                  None if s is None else s.ctypes.data_as(fp)))
    return p, g


def mm_fno_set_output_scale(f, scale):
    _fcheck(_load().mm_fno_set_output_scale(f.handle, float(scale)))


def mm_relax_surrogate(ctx, f, m, t_max, torque_tol=1e-4, max_steps=1000000, k_exact=10, bound=1e-3,
                       torque_exact=0.0):
    """Returns (t, accepted_steps, exact_evals, surrogate_evals, fallbacks)."""
    tt, ss = ctypes.c_double(0.0), ctypes.c_long(0)
    st = (ctypes.c_long * 3)()
    _check(ctx, _load().mm_relax_surrogate(ctx.handle, f.handle, _dev(ctx, m, ctx.shape3, "m"), float(t_max),
                                           float(torque_tol), int(max_steps), int(k_exact), float(bound),
                                           float(torque_exact), ctypes.byref(tt), ctypes.byref(ss), st))
    return tt.value, ss.value, st[0], st[1], st[2]


def relax(ctx, m, t_max, torque_tol=1e-4, max_steps=1000000, surrogate=None, k=10, bound=1e-3, torque_exact=1e-2):
    """relax() of m in place: RKF45 until max |m x H_eff| / Ms <= torque_tol or
    t_max (mm_relax), or with a trained surrogate for the demag field in the
    stages (mm_relax_surrogate: exact field and residual check every k
    steps, exact final approach below torque_exact).  Returns (t, steps)."""
    if surrogate is None:
        return mm_relax(ctx, m, t_max, torque_tol, max_steps)
    t, steps, _, _, _ = mm_relax_surrogate(ctx, surrogate, m, t_max, torque_tol, max_steps, k, bound, torque_exact)
    return t, steps


def from_paper_layout(m_xyz3):
    """(nx, ny, nz, 3) -> (3, nz, ny, nx), the library's component-planar layout."""
    return m_xyz3.permute(3, 2, 1, 0).contiguous() if hasattr(m_xyz3, "permute") else \
        np.ascontiguousarray(np.transpose(m_xyz3, (3, 2, 1, 0)))


def to_paper_layout(m_3zyx):
    """(3, nz, ny, nx) -> (nx, ny, nz, 3)."""
    return m_3zyx.permute(3, 2, 1, 0).contiguous() if hasattr(m_3zyx, "permute") else \
        np.ascontiguousarray(np.transpose(m_3zyx, (3, 2, 1, 0)))
