"""GPU adjoints through the C ABI: transposes of demag and exchange by the
dot-product test, the RK4 step VJP against central differences, whole
trajectories against the oracle's float64 gradient (8 x 8 x 1) and against
the GPU's own central differences on the 256 x 256 x 4 design mesh."""

import numpy as np
import pytest

import workloads as wl
from oracle import adjoint, micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def dev(a, prec=mm.MM_F64):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == mm.MM_F64 else torch.float32,
                        device="cuda")


def vdot(a, b):
    return float(torch.sum(a.double() * b.double()))


def make_ctx(n, d, Ms, prec=mm.MM_F64, Ku=0.0, u=(0, 0, 1), alpha=0.02, h=(0, 0, 0)):
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, alpha, Ku, u)
    mm.mm_set_external_field(ctx, *h)
    mm.mm_set_material_fields(ctx, dev(Ms, prec))
    return ctx


def richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


N_SMALL, D_SMALL = (16, 8, 4), (2.5e-9, 2.5e-9, 3e-9)


def test_demag_transpose_dot_product():
    Ms = wl.smooth_field(N_SMALL, 4e5, 9e5, sigma_cells=2.0, seed=1)
    ctx = make_ctx(N_SMALL, D_SMALL, Ms)
    rng = np.random.default_rng(2)
    v = dev(rng.standard_normal(ctx.shape3))
    g = dev(rng.standard_normal(ctx.shape3))
    Hv = torch.empty_like(v)
    mm.mm_demag_field(ctx, v, Hv)
    gm = torch.empty_like(v)
    gMs = torch.zeros(ctx.shape1, dtype=torch.float64, device="cuda")
    mm.mm_demag_vjp(ctx, g, v, gm, gMs)
    assert vdot(g, Hv) == pytest.approx(vdot(gm, v), rel=1e-12, abs=0)
    # H_d is linear in Ms: the Ms pull-back is exact against a central difference
    delta = dev(rng.standard_normal(ctx.shape1) * 1e4)
    Ms_t = dev(Ms)

    def f(eps):
        mm.mm_set_material_fields(ctx, Ms_t + eps * delta)
        H = torch.empty_like(v)
        mm.mm_demag_field(ctx, v, H)
        return vdot(g, H)
    fd = (f(1.0) - f(-1.0)) / 2.0
    assert fd == pytest.approx(vdot(gMs, delta), rel=1e-10, abs=0)
    mm.mm_destroy(ctx)


def test_exchange_transpose_dot_product_and_ms_gradient():
    Ms = wl.smooth_field(N_SMALL, 4e5, 9e5, sigma_cells=2.0, seed=3)
    ctx = make_ctx(N_SMALL, D_SMALL, Ms)
    rng = np.random.default_rng(4)
    v = dev(rng.standard_normal(ctx.shape3))
    g = dev(rng.standard_normal(ctx.shape3))
    Hv = torch.empty_like(v)
    mm.mm_exchange_field(ctx, v, Hv)
    gm = torch.empty_like(v)
    gMs = torch.zeros(ctx.shape1, dtype=torch.float64, device="cuda")
    mm.mm_exchange_vjp(ctx, g, v, gm, gMs)
    assert vdot(g, Hv) == pytest.approx(vdot(gm, v), rel=1e-12, abs=0)
    delta = dev(rng.standard_normal(ctx.shape1))
    Ms_t = dev(Ms)

    def f(eps):
        mm.mm_set_material_fields(ctx, Ms_t * (1 + eps * delta))
        H = torch.empty_like(v)
        mm.mm_exchange_field(ctx, v, H)
        return vdot(g, H)
    fd = richardson(f, 1e-3)
    assert fd == pytest.approx(vdot(gMs, delta * Ms_t), rel=1e-8, abs=0)
    mm.mm_destroy(ctx)


def test_rk4_step_vjp_against_central_differences():
    Ms = wl.smooth_field(N_SMALL, 4e5, 9e5, sigma_cells=2.0, seed=5)
    ctx = make_ctx(N_SMALL, D_SMALL, Ms, Ku=2e5, u=(0.2, 0.3, 0.9), alpha=0.1, h=(1e4, 0, -2e4))
    rng = np.random.default_rng(6)
    m0 = dev(wl.random_unit(N_SMALL, seed=7))
    lam0 = dev(rng.standard_normal(ctx.shape3))
    v = dev(rng.standard_normal(ctx.shape3))
    delta = dev(rng.standard_normal(ctx.shape1))
    Ms_t = dev(Ms)
    dt = 5e-14
    lam = lam0.clone()
    gMs = torch.zeros(ctx.shape1, dtype=torch.float64, device="cuda")
    mm.mm_rk4_step_vjp(ctx, m0, dt, lam, gMs)

    def step(m, Ms_cell):
        mm.mm_set_material_fields(ctx, Ms_cell)
        x = m.clone()
        mm.mm_llg_step(ctx, x, 0.0, dt, mm.MM_RK4)
        return x

    fm = richardson(lambda e: vdot(lam0, step(m0 + e * v, Ms_t)), 1e-4)
    assert fm == pytest.approx(vdot(lam, v), rel=1e-7, abs=0)
    fs = richardson(lambda e: vdot(lam0, step(m0, Ms_t * (1 + e * delta))), 1e-4)
    assert fs == pytest.approx(vdot(gMs, delta * Ms_t), rel=1e-7, abs=0)
    mm.mm_destroy(ctx)


def _loss(m, target):
    return (m[2].mean() - target) ** 2


def test_trajectory_gradient_matches_oracle_8x8x1():
    """The float64 adjoint of a 40-step RK4 trajectory against the oracle's
    central-difference gradient of the same loss, every cell."""
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    n, d = (8, 8, 1), (3e-9, 3e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=3)
    m0 = wl.random_unit(n, seed=8)
    dt, nsteps, target = 1e-13, 40, 0.05
    ctx = make_ctx(n, d, Ms)
    Ms_t = dev(Ms).requires_grad_(True)
    mN = RK4Trajectory.apply(dev(m0), Ms_t, ctx, dt, nsteps, 7)
    L = _loss(mN, target)
    L.backward()
    g_gpu = Ms_t.grad.detach().cpu().numpy()
    p = micromag.Problem(n, d, Ms_cell=Ms, alpha=0.02)
    g_ref = adjoint.grad_ms(p, m0, dt, nsteps, target).reshape(n[2], n[1], n[0])
    assert float(L.detach()) == pytest.approx(adjoint.loss(p, m0, dt, nsteps, target), rel=1e-10, abs=0)
    assert np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref) < 1e-6
    mm.mm_destroy(ctx)


@pytest.fixture(scope="module")
def design256():
    w = wl.WORKLOADS["design256"]
    Ms = wl.smooth_field(w["n"], 4e5, 9e5, sigma_cells=8.0, seed=3)
    m0 = wl.uniform(w["n"], (1.0, 0.1, 0.3))
    return w, Ms, m0


def test_design256_gradient_central_differences_32_cells(design256):
    """256 x 256 x 4 design mesh, float64 path, 20 RK4 steps: the adjoint's
    dL/dMs at 32 random cells against central differences of the GPU
    forward trajectory."""
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    w, Ms, m0 = design256
    n, d = w["n"], w["d"]
    dt, nsteps, target = 1e-13, 20, 0.05
    ctx = make_ctx(n, d, Ms)
    Ms_t = dev(Ms).requires_grad_(True)
    L = _loss(RK4Trajectory.apply(dev(m0), Ms_t, ctx, dt, nsteps, 0), target)
    L.backward()
    g = Ms_t.grad.detach().cpu().numpy()
    rng = np.random.default_rng(4)
    cells = [(rng.integers(0, n[2]), rng.integers(0, n[1]), rng.integers(0, n[0])) for _ in range(32)]
    base = dev(Ms)
    m0d = dev(m0)

    def loss_at(c, eps):
        Mp = base.clone()
        Mp[c] = Mp[c] * (1 + eps)
        mm.mm_set_material_fields(ctx, Mp)
        m = m0d.clone()
        mm.mm_rk4_trajectory(ctx, m, dt, nsteps)
        return float(_loss(m, target))

    # one cell moves the mean of 262144 cells by ~1e-11 per 1 % of its Ms: the
    # difference quotient carries the loss's roundoff (~1e-16 * L / (h Ms)),
    # about 1e-7 of the gradient scale at h = 1 %, so the bound is 1e-5
    fd = np.array([richardson(lambda e, c=c: loss_at(c, e), 1e-2) / Ms[c] for c in cells])
    ad = np.array([g[c] for c in cells])
    scale = np.max(np.abs(ad))
    assert scale > 0
    assert np.max(np.abs(fd - ad)) / scale < 1e-5
    mm.mm_destroy(ctx)


def test_design256_fp32_adjoint_close_to_fp64(design256):
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    w, Ms, m0 = design256
    n, d = w["n"], w["d"]
    grads = []
    for prec in (mm.MM_F64, mm.MM_F32):
        ctx = make_ctx(n, d, Ms, prec=prec)
        Ms_t = dev(Ms, prec).requires_grad_(True)
        L = _loss(RK4Trajectory.apply(dev(m0, prec), Ms_t, ctx, 1e-13, 100, 0), 0.05)
        L.backward()
        grads.append(Ms_t.grad.detach().double().cpu().numpy())
        mm.mm_destroy(ctx)
    assert np.linalg.norm(grads[1] - grads[0]) / np.linalg.norm(grads[0]) < 1e-3


def test_checkpoint_interval_does_not_change_the_gradient():
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    n, d = (16, 16, 2), (3e-9, 3e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=3.0, seed=9)
    m0 = wl.random_unit(n, seed=10)
    ctx = make_ctx(n, d, Ms)
    out = []
    for k in (1, 5, 0):
        Ms_t = dev(Ms).requires_grad_(True)
        _loss(RK4Trajectory.apply(dev(m0), Ms_t, ctx, 1e-13, 23, k), 0.1).backward()
        out.append(Ms_t.grad.detach().cpu().numpy())
    for o in out[1:]:
        np.testing.assert_allclose(o, out[0], rtol=1e-12, atol=1e-30)
    mm.mm_destroy(ctx)


def test_llg_step_autograd_against_central_differences():
    from paper_2606_01114_gb300.autograd import LLGStep
    Ms = wl.smooth_field(N_SMALL, 4e5, 9e5, sigma_cells=2.0, seed=12)
    ctx = make_ctx(N_SMALL, D_SMALL, Ms, Ku=1e5, u=(0.0, 0.6, 0.8), alpha=0.05)
    rng = np.random.default_rng(13)
    m0 = dev(wl.random_unit(N_SMALL, seed=14)).requires_grad_(True)
    Ms_t = dev(Ms).requires_grad_(True)
    w = dev(rng.standard_normal(ctx.shape3))
    L = torch.sum(w * LLGStep.apply(m0, Ms_t, ctx, 5e-14))
    L.backward()
    v = dev(rng.standard_normal(ctx.shape3))

    def f(e):
        with torch.no_grad():
            return float(torch.sum(w * LLGStep.apply(m0.detach() + e * v, Ms_t.detach(), ctx, 5e-14)))
    assert richardson(f, 1e-4) == pytest.approx(vdot(m0.grad, v), rel=1e-7, abs=0)
    mm.mm_destroy(ctx)


def test_design256_gradient_time_2000_steps(design256):
    """Seconds per gradient on the 256 x 256 x 4 design mesh: 2000 RK4 steps
    of 0.1 ps (0.2 ns) forward and the checkpointed adjoint, float32, with
    the default sqrt(T) checkpoint interval; the gradient is finite and
    non-zero.  The time is printed.  A 2-step gradient runs first: the
    process's first autograd backward pays a one-time start-up of several
    seconds that is not the adjoint's."""
    import time
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    w, Ms, m0 = design256
    ctx = make_ctx(w["n"], w["d"], Ms, prec=mm.MM_F32)
    m0d = dev(m0, mm.MM_F32)
    warm = dev(Ms, mm.MM_F32).requires_grad_(True)
    _loss(RK4Trajectory.apply(m0d, warm, ctx, 1e-13, 2, 0), 0.05).backward()
    Ms_t = dev(Ms, mm.MM_F32).requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mN = RK4Trajectory.apply(m0d, Ms_t, ctx, 1e-13, 2000, 0)
    t1 = time.perf_counter()
    _loss(mN, 0.05).backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = Ms_t.grad
    assert torch.isfinite(g).all() and float(g.abs().max()) > 0
    print(f"design256 float32, 2000 RK4 steps: forward {t1 - t0:.2f} s, gradient (forward + adjoint) {t2 - t0:.2f} s")
    mm.mm_destroy(ctx)


def test_design256_gradient_time_20000_steps_2ns(design256):
    """The differentiation workload at its read horizon: 20,000 RK4 steps of
    0.1 ps (2 ns) forward and the adjoint with sqrt(T) = 142-step
    checkpoints, float32 (memory: 141 checkpoints plus one segment's tape).
    The gradient is finite and non-zero; forward and total times are
    printed."""
    import time
    from paper_2606_01114_gb300.autograd import RK4Trajectory
    w, Ms, m0 = design256
    ctx = make_ctx(w["n"], w["d"], Ms, prec=mm.MM_F32)
    m0d = dev(m0, mm.MM_F32)
    warm = dev(Ms, mm.MM_F32).requires_grad_(True)
    _loss(RK4Trajectory.apply(m0d, warm, ctx, 1e-13, 2, 0), 0.05).backward()
    Ms_t = dev(Ms, mm.MM_F32).requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mN = RK4Trajectory.apply(m0d, Ms_t, ctx, 1e-13, 20000, 0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L = _loss(mN, 0.05)
    L.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = Ms_t.grad
    assert torch.isfinite(g).all() and float(g.abs().max()) > 0
    mz = float(mN[2].mean())
    print(f"design256 float32, 20000 RK4 steps (2 ns): <m_z>(T) = {mz:.6f}, loss {float(L):.3e}, "
          f"forward {t1 - t0:.2f} s, gradient (forward + adjoint) {t2 - t0:.2f} s, "
          f"|dL/dMs| max {float(g.abs().max()):.3e}")
    mm.mm_destroy(ctx)
