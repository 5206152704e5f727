"""Full-size parity on the bench workload: the 512 x 512 x 16 film (padded
FFT grid 1024 x 1024 x 32) that bench.py times, in the launch configuration
it times (the 512-point x passes, the 1024-point y passes and the 32-point
fused z pass).

* The demagnetisation and effective fields over the whole mesh, element by
  element, against the oracle's float64 FFT convolution: relative L2 within
  the path's tolerance (1e-5 FP32, 1e-12 FP64 and float-float), and every
  one of the 12.6 M components within that tolerance times the largest
  component of the field, so that an error confined to some tiles or index
  ranges cannot hide in the norm.
* The first four adaptive RKF45 steps from the bench's start (dt 1e-14 s,
  tol 1e-5) against the oracle's own adaptive trajectory: the same
  accept/reject sequence, the same step sizes (up to the rounding of the
  error estimate) and the same states (float64), or the oracle's step from
  the GPU's state with the GPU's step size (FP32).

The oracle's work (Newell kernel, field, four RKF45 steps) is done once per
process and shared by the cases."""

import functools

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

MODES = {
    "f32": (mm.MM_F32, 0, 1e-5),
    "f64": (mm.MM_F64, 0, 1e-12),
    "ff": (mm.MM_F64, mm.MM_FFT_FF, 1e-12),
    "f4": (mm.MM_F32, mm.MM_FFT_F4, 1e-5),      # the fused y-z-y pass over kx planes
}
RKF45_STEPS = 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def film512():
    w = wl.WORKLOADS["film512"]
    p = micromag.Problem(w["n"], w["d"], Ms=w["Ms"], A=w["A"], alpha=w["alpha"])
    nh = p.kernel_hat()
    p.kernel_hat = lambda: nh          # transform the kernel once
    p._kernel = None                   # the real-space kernel is not needed again
    m = wl.vortex(w["n"], w["d"], noise=0.05, seed=1)
    return p, m


@functools.lru_cache(maxsize=None)
def film512_fields():
    p, m = film512()
    Hd = p.demag_fft(m)
    return Hd, p.h_eff(m, demag=Hd)


@functools.lru_cache(maxsize=None)
def film512_trajectory():
    """The oracle's adaptive RKF45 from the bench's start: per accepted step
    (step size, rejected trials before it, error, state)."""
    p, m = film512()
    t, dt = 0.0, 1e-14
    out = []
    for _ in range(RKF45_STEPS):
        m, t_new, dt, err, rej = micromag.rkf45_step(p, m, t, dt, 1e-5)
        out.append((t_new - t, rej, err, m))
        t = t_new
    return out


def context(mode):
    prec, fft_mode, _ = MODES[mode]
    p, _ = film512()
    ctx = mm.mm_init_mesh(*p.n, *p.d, precision=prec)
    mm.mm_set_material(ctx, float(p.Ms.flat[0]), float(p.A.flat[0]), p.alpha, 0.0)
    if fft_mode:
        mm.mm_set_fft_mode(ctx, fft_mode)
    return ctx


def dev(a, mode):
    dt = torch.float32 if MODES[mode][0] == mm.MM_F32 else torch.float64
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def check_elementwise(got, ref, tol, what):
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    err = np.abs(got - ref)
    worst = np.unravel_index(int(np.argmax(err)), err.shape)
    bound = tol * float(np.max(np.abs(ref)))
    assert rel < tol, f"{what}: relative L2 {rel:.3e}"
    assert err[worst] <= bound, (f"{what}: component {worst[0]} at (z, y, x) = {worst[1:]} is off by "
                                 f"{err[worst]:.3e} > {bound:.3e}")
    return rel, float(err[worst]) / float(np.max(np.abs(ref)))


@pytest.mark.parametrize("mode", list(MODES))
def test_film512_demag_and_effective_field_every_cell(mode):
    _, _, tol = MODES[mode]
    p, m = film512()
    Hd_ref, He_ref = film512_fields()
    ctx = context(mode)
    md = dev(m, mode)
    H = torch.empty_like(md)
    mm.mm_demag_field(ctx, md, H)
    rd = check_elementwise(host(H), Hd_ref, tol, "demag")
    mm.mm_effective_field(ctx, md, H)
    re = check_elementwise(host(H), He_ref, tol, "effective field")
    print(f"film512 {mode}: demag rel-L2 {rd[0]:.2e}, max element {rd[1]:.2e}; "
          f"effective rel-L2 {re[0]:.2e}, max element {re[1]:.2e}")
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("mode", list(MODES))
def test_film512_rkf45_first_steps_match_oracle_trajectory(mode):
    prec, _, tol = MODES[mode]
    p, m0 = film512()
    ref = film512_trajectory()
    ctx = context(mode)
    md = dev(m0, mode)
    t, dt = 0.0, 1e-14
    # Step sizes follow the error estimate through the controller, so they
    # agree to the estimate's rounding.  Float64 estimates agree to ~1e-10.
    # In FP32 the first estimate (6e-9, a difference of stage slopes ~1e5
    # times smaller than the state change) carries ~1 % rounding, which the
    # controller's fifth root turns into ~0.3 % of the next step size; so the
    # FP32 states are checked step by step against the oracle's trial from the
    # GPU's previous state with the GPU's step size, the float64 states
    # against the oracle's own trajectory.
    h_tol = 1e-2 if prec == mm.MM_F32 else 1e-8
    for i, (h_ref, rej_ref, err_ref, m_ref) in enumerate(ref):
        m_prev = host(md)
        t_new, dt_next, err = mm.mm_llg_step(ctx, md, t, dt, mm.MM_RKF45, tol=1e-5)
        _, rej, _, _ = mm.mm_step_stats(ctx)
        h = t_new - t
        assert rej == rej_ref, f"step {i}: {rej} rejected trials, oracle {rej_ref}"
        assert h == pytest.approx(h_ref, rel=h_tol, abs=0), f"step {i}"
        assert err <= 1e-5
        assert dt_next == pytest.approx(micromag.next_dt(h, err, 1e-5), rel=1e-9, abs=0)
        got = host(md)
        if prec == mm.MM_F32:
            m_loc, _ = p.rkf45_trial(m_prev, h)
            rel = float(np.linalg.norm(got - m_loc) / np.linalg.norm(m_loc))
        else:
            rel = float(np.linalg.norm(got - m_ref) / np.linalg.norm(m_ref))
        assert rel < tol, f"step {i}: state rel-L2 {rel:.3e}"
        print(f"film512 {mode} step {i}: h {h:.4e} (oracle {h_ref:.4e}), rejected {rej}, "
              f"err {err:.3e} (oracle {err_ref:.3e}), state rel-L2 {rel:.2e}")
        t, dt = t_new, dt_next
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("n", [(16, 512, 16), (40, 512, 16)])
def test_fused_yzy_pass_on_narrow_films_matches_oracle(n):
    """MM_FFT_F4 on meshes of the supported ny and nz with few x cells (a
    power of two and a direct-DFT x length): demag against the oracle,
    element by element."""
    d = (2e-9, 2e-9, 2e-9)
    p = micromag.Problem(n, d)
    m = wl.random_unit(n, seed=12)
    ctx = mm.mm_init_mesh(*n, *d, precision=mm.MM_F32)
    mm.mm_set_fft_mode(ctx, mm.MM_FFT_F4)
    md = torch.tensor(m, dtype=torch.float32, device="cuda")
    H = torch.empty_like(md)
    mm.mm_demag_field(ctx, md, H)
    check_elementwise(host(H), p.demag_fft(m), 1e-5, "demag")
    mm.mm_destroy(ctx)


def test_fused_yzy_pass_rejects_other_meshes():
    for n, prec in (((64, 256, 16), mm.MM_F32), ((64, 512, 8), mm.MM_F32), ((64, 512, 16), mm.MM_F64)):
        ctx = mm.mm_init_mesh(*n, 2e-9, 2e-9, 2e-9, precision=prec)
        with pytest.raises(mm.MMError) as e:
            mm.mm_set_fft_mode(ctx, mm.MM_FFT_F4)
        assert e.value.code == mm.MM_ERR_INVALID_ARG
        mm.mm_destroy(ctx)
