"""GPU parity of the float-float mode (MM_FFT_FF on an MM_F64 context: the
demag passes, and for uniform material the stage kernel, in float-float
arithmetic) against the float64 CPU oracle, at the float64 path's tolerance
(relative L2 1e-12 per field): demag on the power-of-two meshes of the main
parity suite, per-cell Ms with vacuum, a 128 x 128 x 16 film, RK4 steps
checked one by one, an RKF45 trial (state, error estimate, proposal) and a
rejected-then-accepted step, the transpose (dot-product) test of the
adjoint, and the mode's error paths."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ff_ctx(p, mode=mm.MM_FFT_FF):
    nx, ny, nz = p.n
    ctx = mm.mm_init_mesh(nx, ny, nz, *p.d, precision=mm.MM_F64)
    uniform = np.all(p.Ms == p.Ms.flat[0])
    mm.mm_set_material(ctx, float(p.Ms.flat[0]) if uniform else 8e5, float(p.A.flat[0]), p.alpha, p.Ku, tuple(p.u))
    mm.mm_set_external_field(ctx, *p.h_ext)
    if not uniform:
        mm.mm_set_material_fields(ctx, dev(p.Ms))
    mm.mm_set_fft_mode(ctx, mode)
    return ctx


MESHES = [
    ((8, 4, 2), (2.5e-9, 2.5e-9, 3e-9)),
    ((16, 8, 1), (2e-9, 2e-9, 2e-9)),
    ((1, 8, 4), (2e-9, 1e-9, 3e-9)),
    ((4, 1, 1), (1e-9, 1e-9, 1e-9)),
    ((32, 16, 8), (2e-9, 2e-9, 2e-9)),
    ((64, 64, 4), (2.5e-9, 2.5e-9, 3e-9)),
    ((128, 128, 16), (2e-9, 2e-9, 2e-9)),
]


@pytest.mark.parametrize("n,d", MESHES)
def test_ff_demag_matches_oracle(n, d):
    p = micromag.Problem(n, d)
    m = wl.random_unit(n, seed=0)
    ctx = ff_ctx(p)
    H = torch.empty(ctx.shape3, dtype=torch.float64, device="cuda")
    mm.mm_demag_field(ctx, dev(m), H)
    err = rel_l2(host(H), p.demag_fft(m))
    assert err < TOL, err
    mm.mm_destroy(ctx)


def test_ff_demag_per_cell_ms_with_vacuum():
    n, d = (32, 16, 4), (2e-9, 3e-9, 1.5e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=3.0, seed=5)
    Ms[:, :4, :5] = 0.0
    p = micromag.Problem(n, d, Ms_cell=Ms)
    m = wl.random_unit(n, seed=1)
    ctx = ff_ctx(p)
    H = torch.empty(ctx.shape3, dtype=torch.float64, device="cuda")
    mm.mm_demag_field(ctx, dev(m), H)
    assert rel_l2(host(H), p.demag_fft(m)) < TOL
    mm.mm_destroy(ctx)


def test_ff_rk4_steps_film64():
    """64 x 64 x 4 film, random m, 20 RK4 steps at 1e-13 s: each GPU step
    against the oracle's step from the GPU's previous state (1e-12), and
    |m| = 1 after every step."""
    w = wl.WORKLOADS["film64"]
    p = micromag.Problem(w["n"], w["d"], Ms=w["Ms"], A=w["A"], alpha=w["alpha"])
    m = wl.random_unit(w["n"], seed=0)
    ctx = ff_ctx(p)
    md = dev(m)
    t = 0.0
    prev = m
    for _ in range(20):
        t, _, _ = mm.mm_llg_step(ctx, md, t, 1e-13, mm.MM_RK4)
        cur = host(md)
        assert rel_l2(cur, p.rk4_step(prev, 1e-13)) < TOL
        assert np.max(np.abs(np.linalg.norm(cur, axis=0) - 1)) < 1e-14
        prev = cur
    mm.mm_destroy(ctx)


def test_ff_demag_transpose_dot_product():
    """Demag with the symmetric Newell tensor is self-adjoint:
    <g, H(v)> = <H(g), v> through the adjoint entry point, to 1e-12."""
    n, d = (16, 8, 4), (2.5e-9, 2.5e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=1)
    p = micromag.Problem(n, d, Ms_cell=Ms)
    ctx = ff_ctx(p)
    rng = np.random.default_rng(2)
    v = dev(rng.standard_normal(ctx.shape3))
    g = dev(rng.standard_normal(ctx.shape3))
    Hv = torch.empty_like(v)
    mm.mm_demag_field(ctx, v, Hv)
    gm = torch.empty_like(v)
    gMs = torch.zeros(ctx.shape1, dtype=torch.float64, device="cuda")
    mm.mm_demag_vjp(ctx, g, v, gm, gMs)
    a, b = float(torch.sum(g * Hv)), float(torch.sum(gm * v))
    assert a == pytest.approx(b, rel=1e-12, abs=0)
    mm.mm_destroy(ctx)


def test_ff_mode_switches_back_to_native():
    """Mode 0 after MM_FFT_FF gives the native float64 field again, and both
    agree with the oracle."""
    n, d = (32, 16, 8), (2e-9, 2e-9, 2e-9)
    p = micromag.Problem(n, d)
    m = dev(wl.random_unit(n, seed=3))
    ctx = ff_ctx(p)
    H_ff = torch.empty_like(m)
    mm.mm_demag_field(ctx, m, H_ff)
    mm.mm_set_fft_mode(ctx, 0)
    H_64 = torch.empty_like(m)
    mm.mm_demag_field(ctx, m, H_64)
    ref = p.demag_fft(host(m))
    assert rel_l2(host(H_ff), ref) < TOL
    assert rel_l2(host(H_64), ref) < TOL
    assert not torch.equal(H_ff, H_64)          # the two arithmetics really differ
    mm.mm_destroy(ctx)


def test_ff_mode_errors():
    ctx = mm.mm_init_mesh(8, 8, 2, 1e-9, 1e-9, 1e-9, precision=mm.MM_F32)
    with pytest.raises(mm.MMError) as e:
        mm.mm_set_fft_mode(ctx, mm.MM_FFT_FF)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    mm.mm_destroy(ctx)
    ctx = mm.mm_init_mesh(100, 25, 1, 5e-9, 5e-9, 3e-9, precision=mm.MM_F64)   # Px = 200
    with pytest.raises(mm.MMError) as e:
        mm.mm_set_fft_mode(ctx, mm.MM_FFT_FF)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    mm.mm_destroy(ctx)


def _rkf45_error_bound(p, m, dt, unit_roundoff):
    """Rounding bound of the embedded error estimate dt |sum_j e_j k_j|: the
    stage slopes carry a relative error of order the unit roundoff, so the
    estimate is uncertain by about u * dt * max_cell sum_j |e_j| |k_j|."""
    k = []
    for s in range(6):
        ms = m.copy()
        for j in range(s):
            ms = ms + dt * micromag.FEHLBERG_A[s][j] * k[j]
        k.append(p.rhs(ms))
    e = [b5 - b4 for b5, b4 in zip(micromag.FEHLBERG_B5, micromag.FEHLBERG_B4)]
    mag = sum(abs(e[j]) * np.sqrt(np.sum(k[j] ** 2, axis=0)) for j in range(6))
    return unit_roundoff * dt * float(np.max(mag))


def test_ff_rkf45_trial_matches_oracle():
    """One RKF45 trial with the float-float stage kernel (uniform material):
    the 4th-order state at 1e-12, the error estimate within the float-float
    rounding bound (unit roundoff 2^-48), and the controller's proposal."""
    n, d = (16, 16, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=0.1, Ku=2e5, u=(0, 0, 1), h_ext=(2e4, 0, 0))
    m = wl.random_unit(n, seed=4)
    ctx = ff_ctx(p)
    md = dev(m)
    dt = 2e-14
    t, dt_next, err = mm.mm_llg_step(ctx, md, 0.0, dt, mm.MM_RKF45, tol=1.0)   # accepted at any error
    m4, err_o = p.rkf45_trial(m, dt)
    assert t == dt
    assert rel_l2(host(md), m4) < TOL
    assert np.max(np.abs(np.linalg.norm(host(md), axis=0) - 1)) < 1e-14
    assert abs(err - err_o) < 8 * _rkf45_error_bound(p, m, dt, 2.0 ** -48) + 1e-9 * err_o
    assert dt_next == pytest.approx(micromag.next_dt(dt, err, 1.0), rel=1e-12, abs=0)
    mm.mm_destroy(ctx)


def test_ff_rkf45_rejects_then_accepts():
    n, d = (8, 8, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=0.02, Ku=1e5, u=(0.0, 0.6, 0.8), h_ext=(1e4, 0.0, -2e4))
    m = wl.random_unit(n, seed=11)
    ctx = ff_ctx(p)
    md = dev(m)
    t, dt_next, err = mm.mm_llg_step(ctx, md, 0.0, 1e-11, mm.MM_RKF45, tol=1e-5)
    mo, to, dto, erro, rej = micromag.rkf45_step(p, m, 0.0, 1e-11, 1e-5)
    assert rej >= 1
    assert t == pytest.approx(to, rel=1e-12, abs=0)
    assert err <= 1e-5
    assert rel_l2(host(md), mo) < TOL
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("case", ["dmi", "per_cell_ms"])
def test_ff_rk4_steps_with_the_fp64_stage(case):
    """Materials outside the float-float stage kernel (interfacial DMI; per-cell
    Ms) keep the float64 stage beside the float-float demag
    passes: 15 RK4 steps, each against the oracle's step from the GPU's
    previous state at 1e-12."""
    n, d = (16, 16, 2), (2.5e-9, 2.5e-9, 2.5e-9)
    if case == "dmi":
        p = micromag.Problem(n, d, alpha=0.1, D=4e-3, dmi="interfacial")
    else:
        Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=7)
        p = micromag.Problem(n, d, alpha=0.1, Ms_cell=Ms)
    ctx = ff_ctx(p)
    if case == "dmi":
        mm.mm_set_dmi(ctx, 4e-3, mm.MM_DMI_INTERFACIAL)
    m = wl.random_unit(n, seed=6)
    md = dev(m)
    prev, t = m, 0.0
    for _ in range(15):
        t, _, _ = mm.mm_llg_step(ctx, md, t, 5e-14, mm.MM_RK4)
        cur = host(md)
        assert rel_l2(cur, p.rk4_step(prev, 5e-14)) < TOL
        prev = cur
    mm.mm_destroy(ctx)


def test_ff_demag_film512_sampled_cells():
    """The bench workload at full size (512 x 512 x 16 film, vortex with 5 %
    noise) in float-float mode: 8 sampled cells against the oracle's direct
    sum over all 4.2 M sources, at the float64 tolerance."""
    w = wl.WORKLOADS["film512"]
    p = micromag.Problem(w["n"], w["d"], Ms=w["Ms"], A=w["A"], alpha=w["alpha"])
    m = wl.vortex(w["n"], w["d"], noise=0.05, seed=1)
    ctx = ff_ctx(p)
    H = torch.empty(ctx.shape3, dtype=torch.float64, device="cuda")
    mm.mm_demag_field(ctx, dev(m), H)
    got = host(H)
    targets = [(0, 0, 0), (511, 511, 15), (256, 256, 8), (255, 256, 0), (0, 300, 7), (511, 17, 3),
               (100, 400, 15), (383, 129, 9)]
    ref = p.demag_direct(m, targets)
    sel = np.stack([got[:, z, y, x] for (x, y, z) in targets], axis=1)
    assert rel_l2(sel, ref) < TOL
    mm.mm_destroy(ctx)


def test_ff_trajectory_gradient_matches_oracle_8x8x1():
    """The adjoint of a 40-step RK4 trajectory with the float-float demag
    passes (forward, replay and transposed demag all in float-float) against
    the oracle's float64 gradient of the same loss, every cell."""
    from oracle import adjoint
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    n, d = (8, 8, 1), (3e-9, 3e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=3)
    m0 = wl.random_unit(n, seed=8)
    dt, nsteps, target = 1e-13, 40, 0.05
    p = micromag.Problem(n, d, Ms_cell=Ms, alpha=0.02)
    ctx = ff_ctx(p)
    Ms_t = dev(Ms).requires_grad_(True)
    mN = RK4Trajectory.apply(dev(m0), Ms_t, ctx, dt, nsteps, 7)
    L = (mN[2].mean() - target) ** 2
    L.backward()
    g_gpu = Ms_t.grad.detach().cpu().numpy()
    g_ref = adjoint.grad_ms(p, m0, dt, nsteps, target).reshape(n[2], n[1], n[0])
    assert float(L.detach()) == pytest.approx(adjoint.loss(p, m0, dt, nsteps, target), rel=1e-10, abs=0)
    assert np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref) < 1e-6
    mm.mm_destroy(ctx)
