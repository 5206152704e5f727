"""GPU parity: every step of the hot path through the C ABI against the CPU
oracle on the same seeded inputs.  Tolerances (relative L2 per field):
1e-12 for the float64 path, 1e-5 for the float32 path."""

import functools
import os

import numpy as np
import pytest

import workloads as wl
from oracle import micromag, newell

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {mm.MM_F64: 1e-12, mm.MM_F32: 1e-5}
PRECS = [mm.MM_F64, mm.MM_F32]
PNAME = {mm.MM_F64: "f64", mm.MM_F32: "f32"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def dev(a, prec):
    dt = torch.float64 if prec == mm.MM_F64 else torch.float32
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def oracle_problem(n, d, Ms=8e5, A=1.3e-11, alpha=0.02, Ku=0.0, seed_ms=None):
    Ms_cell = None
    if seed_ms is not None:
        Ms_cell = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=seed_ms)
    return micromag.Problem(n, d, Ms=Ms, A=A, alpha=alpha, Ku=Ku, Ms_cell=Ms_cell)


def gpu_ctx(p, prec):
    nx, ny, nz = p.n
    ctx = mm.mm_init_mesh(nx, ny, nz, *p.d, precision=prec)
    uniform_ms = float(p.Ms.flat[0]) if np.all(p.Ms == p.Ms.flat[0]) else 8e5
    mm.mm_set_material(ctx, uniform_ms, float(p.A.flat[0]), p.alpha, p.Ku, tuple(p.u))
    mm.mm_set_external_field(ctx, *p.h_ext)
    if not np.all(p.Ms == p.Ms.flat[0]):
        ms = dev(p.Ms, prec)
        A = dev(p.A, prec) if not np.all(p.A == p.A.flat[0]) else None
        mm.mm_set_material_fields(ctx, ms, A)
    return ctx


MESHES = [
    ((8, 4, 2), (2.5e-9, 2.5e-9, 3e-9)),
    ((16, 8, 1), (2e-9, 2e-9, 2e-9)),
    ((1, 8, 4), (2e-9, 1e-9, 3e-9)),
    ((4, 1, 1), (1e-9, 1e-9, 1e-9)),
    ((32, 16, 8), (2e-9, 2e-9, 2e-9)),
    ((64, 64, 4), (2.5e-9, 2.5e-9, 3e-9)),
]


@pytest.mark.parametrize("n,d", MESHES + [((32, 8, 1), (4e-9, 4e-9, 0.7e-9)), ((16, 16, 16), (1e-9, 1e-9, 1e-9))])
def test_newell_tensor_matches_oracle(n, d):
    p = oracle_problem(n, d)
    ctx = gpu_ctx(p, mm.MM_F64)
    got = mm.mm_newell_tensor(ctx)
    ref = newell.kernel_octant(n, d)
    assert np.max(np.abs(got - ref)) < 2e-16
    assert rel_l2(got, ref) < 1e-14
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("n,d", MESHES)
def test_demag_matches_oracle(n, d, prec):
    p = oracle_problem(n, d)
    m = wl.random_unit(n, seed=0)
    ctx = gpu_ctx(p, prec)
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    mm.mm_demag_field(ctx, dev(m, prec), H)
    assert rel_l2(host(H), p.demag_fft(m)) < TOL[prec]
    mm.mm_destroy(ctx)


# Py = 1024 and 512 take the TMA-fed y passes in FP32 (8-column tiles, the
# last one ragged: Hx = 25 and 41); the x passes here are the direct-DFT
# (Px = 48) and Bluestein (Px = 80) ones, and nz = 1 takes the Pz = 1 z pass.
# nx = 512 takes the TMA-fed x passes (4-row tiles; 3 x 1 x 3 = 9 rows leave
# a last tile of one row)
TMA_Y_MESHES = [
    ((24, 512, 2), (2e-9, 2e-9, 3e-9)),
    ((40, 256, 4), (3e-9, 2e-9, 2e-9)),
    ((16, 512, 1), (2e-9, 2e-9, 1e-9)),
    ((512, 8, 2), (2e-9, 2e-9, 3e-9)),
    ((512, 3, 1), (2e-9, 3e-9, 2e-9)),
]


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("n,d", TMA_Y_MESHES)
def test_demag_tma_y_pass_meshes_match_oracle(n, d, prec):
    p = oracle_problem(n, d)
    m = wl.random_unit(n, seed=7)
    ctx = gpu_ctx(p, prec)
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    mm.mm_demag_field(ctx, dev(m, prec), H)
    got, ref = host(H), p.demag_fft(m)
    assert rel_l2(got, ref) < TOL[prec]
    # every cell, against the field's scale
    assert np.max(np.abs(got - ref)) < 10 * TOL[prec] * np.max(np.abs(ref))
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_demag_per_cell_ms_with_vacuum(prec):
    n, d = (32, 16, 4), (2e-9, 3e-9, 1.5e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=3.0, seed=5)
    Ms[:, :4, :5] = 0.0
    p = micromag.Problem(n, d, Ms_cell=Ms)
    m = wl.random_unit(n, seed=1)
    ctx = gpu_ctx(p, prec)
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    mm.mm_demag_field(ctx, dev(m, prec), H)
    assert rel_l2(host(H), p.demag_fft(m)) < TOL[prec]
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_exchange_and_effective_field(prec):
    n, d = (16, 8, 4), (2e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(3)
    Ms = rng.uniform(4e5, 9e5, size=(4, 8, 16))
    Ms[1, 2, 3] = 0.0
    Ms[3, 7, 15] = 0.0
    A = rng.uniform(0.5e-11, 2e-11, size=(4, 8, 16))
    p = micromag.Problem(n, d, Ms_cell=Ms, A_cell=A, Ku=3e5, u=(0.3, -0.2, 0.9), h_ext=(1e4, -2e4, 3e4))
    m = wl.random_unit(n, seed=2)
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.02, 3e5, (0.3, -0.2, 0.9))
    mm.mm_set_external_field(ctx, 1e4, -2e4, 3e4)
    mm.mm_set_material_fields(ctx, dev(Ms, prec), dev(A, prec))
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    md = dev(m, prec)
    mm.mm_exchange_field(ctx, md, H)
    assert rel_l2(host(H), p.exchange(m)) < TOL[prec]
    mm.mm_effective_field(ctx, md, H)
    assert rel_l2(host(H), p.h_eff(m)) < TOL[prec]
    E = mm.mm_energy(ctx, md)
    Eo = p.energies(m)
    scale = np.sum(np.abs(Eo))
    assert np.max(np.abs(E - Eo)) / scale < TOL[prec]
    tq = mm.mm_max_torque(ctx, md)
    assert tq == pytest.approx(p.max_torque(m), rel=10 * TOL[prec], abs=0)
    mm.mm_destroy(ctx)


# uniform material, nx a multiple of 4: the four-cell FP32 field kernels
# (x edges inside and across the quads, one-cell-thick axes); FP64 takes the
# generic kernel on the same inputs
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("n,d", [((16, 8, 4), (2e-9, 2.5e-9, 3e-9)), ((4, 6, 1), (2e-9, 2e-9, 2e-9)),
                                 ((64, 32, 2), (3e-9, 2e-9, 4e-9))])
def test_exchange_and_effective_field_uniform_material(n, d, prec):
    p = micromag.Problem(n, d, Ku=3e5, u=(0.3, -0.2, 0.9), h_ext=(1e4, -2e4, 3e4))
    m = wl.random_unit(n, seed=9)
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.02, 3e5, (0.3, -0.2, 0.9))
    mm.mm_set_external_field(ctx, 1e4, -2e4, 3e4)
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    md = dev(m, prec)
    mm.mm_exchange_field(ctx, md, H)
    got, ref = host(H), p.exchange(m)
    assert rel_l2(got, ref) < TOL[prec]
    assert np.max(np.abs(got - ref)) < 10 * TOL[prec] * np.max(np.abs(ref))
    mm.mm_effective_field(ctx, md, H)
    assert rel_l2(host(H), p.h_eff(m)) < TOL[prec]
    mm.mm_destroy(ctx)


def test_rk4_film64_200_steps_fp64():
    """64 x 64 x 4 permalloy film, random m, 200 RK4 steps at dt = 1e-13 s.

    Every step is checked locally (the oracle's step from the GPU's previous
    state, 1e-12).  The whole trajectory is checked against the oracle's own
    trajectory within 3e-9: random spins make this flow unstable, and a
    1-ulp perturbation of the initial state alone grows to 2.7e-10 after 200
    oracle steps (about 7 % per step after the first 50), so no bound below
    that can hold for two correct float64 programs."""
    w = wl.WORKLOADS["film64"]
    p = oracle_problem(w["n"], w["d"], Ms=w["Ms"], A=w["A"], alpha=w["alpha"])
    m0 = wl.random_unit(w["n"], seed=0)
    ctx = gpu_ctx(p, mm.MM_F64)
    md = dev(m0, mm.MM_F64)
    H = torch.empty(ctx.shape3, dtype=torch.float64, device="cuda")
    mm.mm_demag_field(ctx, md, H)
    assert rel_l2(host(H), p.demag_fft(m0)) < 1e-12
    mm.mm_exchange_field(ctx, md, H)
    assert rel_l2(host(H), p.exchange(m0)) < 1e-12
    t = 0.0
    m = m0.copy()
    prev = m0.copy()
    worst = 0.0
    for _ in range(200):
        t, _, _ = mm.mm_llg_step(ctx, md, t, 1e-13, mm.MM_RK4)
        cur = host(md)
        worst = max(worst, rel_l2(cur, p.rk4_step(prev, 1e-13)))
        prev = cur
        m = p.rk4_step(m, 1e-13)
    assert worst < 1e-12
    assert t == pytest.approx(200 * 1e-13, rel=1e-12, abs=0)
    assert rel_l2(prev, m) < 3e-9
    assert np.max(np.abs(np.linalg.norm(prev, axis=0) - 1)) < 1e-14
    mm.mm_destroy(ctx)


def test_rk4_film64_20_steps_fp32():
    w = wl.WORKLOADS["film64"]
    p = oracle_problem(w["n"], w["d"], Ms=w["Ms"], A=w["A"], alpha=w["alpha"])
    m = wl.random_unit(w["n"], seed=0)
    ctx = gpu_ctx(p, mm.MM_F32)
    md = dev(m, mm.MM_F32)
    t = 0.0
    prev = host(md)
    for _ in range(20):
        t, _, _ = mm.mm_llg_step(ctx, md, t, 1e-13, mm.MM_RK4)
        cur = host(md)
        assert rel_l2(cur, p.rk4_step(prev, 1e-13)) < 1e-5
        prev = cur
        m = p.rk4_step(m, 1e-13)
    assert rel_l2(prev, m) < 1e-5
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


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_rkf45_trial_matches_oracle(prec):
    n, d = (16, 16, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=0.1, Ku=2e5, u=(0, 0, 1), h_ext=(2e4, 0, 0))
    m = wl.random_unit(n, seed=4)
    ctx = gpu_ctx(p, prec)
    md = dev(m, prec)
    dt = 2e-14
    t, dt_next, err = mm.mm_llg_step(ctx, md, 0.0, dt, mm.MM_RKF45, tol=1.0)   # accepted at any error
    m4, err_o = p.rkf45_trial(m, dt)
    assert t == dt
    assert rel_l2(host(md), m4) < TOL[prec]
    u = 2.0 ** -53 if prec == mm.MM_F64 else 2.0 ** -24
    assert abs(err - err_o) < 8 * _rkf45_error_bound(p, m, dt, u) + 1e-9 * err_o
    assert dt_next == pytest.approx(micromag.next_dt(dt, err, 1.0), rel=1e-12, abs=0)
    mm.mm_destroy(ctx)


def test_rkf45_rejects_then_accepts_fp64():
    n, d = (8, 8, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=0.02, Ku=1e5, u=(0.0, 0.6, 0.8), h_ext=(1e4, 0.0, -2e4))
    m = wl.random_unit(n, seed=11)
    ctx = gpu_ctx(p, mm.MM_F64)
    md = dev(m, mm.MM_F64)
    t, dt_next, err = mm.mm_llg_step(ctx, md, 0.0, 1e-11, mm.MM_RKF45, tol=1e-5)
    mo, to, dto, erro, rej = micromag.rkf45_step(p, m, 0.0, 1e-11, 1e-5)
    assert rej >= 1
    assert t == pytest.approx(to, rel=1e-12, abs=0)
    assert err <= 1e-5
    assert rel_l2(host(md), mo) < 1e-12
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_rkf45_trajectory_replayed_by_the_oracle(prec):
    """Adaptive RKF45 on the GPU for 40 accepted steps; the oracle replays
    the GPU's accepted step sizes (rkf45_trial with each dt) and the states
    agree step by step, while every proposed next step follows the
    controller formula from the GPU's own error."""
    n, d = (16, 16, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=0.1, Ku=2e5, u=(0, 0, 1), h_ext=(2e4, 0, 0))
    m = wl.random_unit(n, seed=21)
    ctx = gpu_ctx(p, prec)
    md = dev(m, prec)
    t, dt = 0.0, 1e-14
    worst = 0.0
    for _ in range(40):
        t_new, dt_next, err = mm.mm_llg_step(ctx, md, t, dt, mm.MM_RKF45, tol=1e-5)
        h = t_new - t
        m, err_o = p.rkf45_trial(m, h)
        worst = max(worst, rel_l2(host(md), m))
        assert err <= 1e-5
        assert dt_next == pytest.approx(micromag.next_dt(h, err, 1e-5), rel=1e-9, abs=0)
        t, dt = t_new, dt_next
    assert worst < (1e-12 if prec == mm.MM_F64 else 2e-5), worst
    mm.mm_destroy(ctx)


def test_relax_macrospin_aligns_with_field():
    p = micromag.Problem((1, 1, 1), (2e-9, 2e-9, 2e-9), alpha=0.5, h_ext=(0, 0, 3e5))
    m = np.array([np.sin(1.0) * np.cos(0.3), np.sin(1.0) * np.sin(0.3), np.cos(1.0)]).reshape(3, 1, 1, 1)
    ctx = gpu_ctx(p, mm.MM_F64)
    md = dev(m, mm.MM_F64)
    t, steps = mm.mm_relax(ctx, md, t_max=5e-9, torque_tol=1e-4, max_steps=100000)
    assert t < 5e-9 and steps > 0
    assert mm.mm_max_torque(ctx, md) <= 1e-4
    assert host(md)[2, 0, 0, 0] > 1 - 1e-7
    mm.mm_destroy(ctx)


def test_relax_film_energy_decreases_fp32():
    n, d = (64, 64, 2), (2.5e-9, 2.5e-9, 3e-9)
    m = wl.vortex(n, d, core_radius=8e-9, noise=0.05, seed=1)
    ctx = mm.mm_init_mesh(*n, *d, precision=mm.MM_F32)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.5, 0.0)
    md = dev(m, mm.MM_F32)
    E0 = mm.mm_energy(ctx, md).sum()
    t, steps = mm.mm_relax(ctx, md, t_max=2e-11, torque_tol=0.0, max_steps=100000)
    E1 = mm.mm_energy(ctx, md).sum()
    assert t == pytest.approx(2e-11, rel=1e-9, abs=0)
    assert E1 < E0
    got = host(md)
    assert np.max(np.abs(np.linalg.norm(got, axis=0) - 1)) < 1e-6
    mm.mm_destroy(ctx)


def test_nonfinite_input_is_reported():
    ctx = mm.mm_init_mesh(8, 8, 1, 2e-9, 2e-9, 2e-9, precision=mm.MM_F32)
    m = wl.random_unit((8, 8, 1), seed=0)
    m[0, 0, 3, 3] = np.nan
    md = dev(m, mm.MM_F32)
    with pytest.raises(mm.MMError) as e:
        mm.mm_llg_step(ctx, md, 0.0, 1e-13, mm.MM_RK4)
    assert e.value.code == mm.MM_ERR_NONFINITE
    # the context stays usable
    md = dev(wl.random_unit((8, 8, 1), seed=0), mm.MM_F32)
    mm.mm_llg_step(ctx, md, 0.0, 1e-13, mm.MM_RK4)
    mm.mm_destroy(ctx)


def test_save_load_roundtrip(tmp_path):
    ctx = mm.mm_init_mesh(8, 4, 2, 2e-9, 2e-9, 2e-9, precision=mm.MM_F64)
    m = dev(wl.random_unit((8, 4, 2), seed=9), mm.MM_F64)
    path = os.path.join(tmp_path, "state.bin")
    mm.mm_save_state(ctx, m, 1.5e-12, 3e-14, path)
    m2 = torch.zeros_like(m)
    t, dt = mm.mm_load_state(ctx, m2, path)
    assert (t, dt) == (1.5e-12, 3e-14)
    assert torch.equal(m, m2)
    other = mm.mm_init_mesh(4, 4, 2, 2e-9, 2e-9, 2e-9, precision=mm.MM_F64)
    with pytest.raises(mm.MMError):
        mm.mm_load_state(other, torch.zeros((3, 2, 4, 4), dtype=torch.float64, device="cuda"), path)
    mm.mm_destroy(ctx)
    mm.mm_destroy(other)


@functools.lru_cache(maxsize=None)
def film512_problem():
    w = wl.WORKLOADS["film512"]
    return micromag.Problem(w["n"], w["d"], Ms=w["Ms"], A=w["A"], alpha=w["alpha"])


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_demag_film512_sampled_cells(prec):
    """512 x 512 x 16 film (the bench workload): sampled cells against the
    oracle's direct sum over all 4.2 M sources."""
    w = wl.WORKLOADS["film512"]
    p = film512_problem()
    m = wl.vortex(w["n"], w["d"], noise=0.05, seed=1)
    ctx = gpu_ctx(p, prec)
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    mm.mm_demag_field(ctx, dev(m, prec), H)
    got = host(H)
    targets = [(0, 0, 0), (511, 511, 15), (256, 256, 8), (255, 256, 0), (0, 300, 7), (511, 17, 3),
               (100, 400, 15), (383, 129, 9)]
    ref = p.demag_direct(m, targets)
    sel = np.stack([got[:, z, y, x] for (x, y, z) in targets], axis=1)
    assert rel_l2(sel, ref) < TOL[prec]
    mm.mm_destroy(ctx)


def test_error_paths_underflow_and_step_cap():
    """RKF45 with an unreachable tolerance shrinks dt below 1e-20 s and
    reports DT_UNDERFLOW; relax() that hits max_steps first reports
    NOT_CONVERGED; both leave the context usable."""
    n, d = (8, 8, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=0.02)
    ctx = gpu_ctx(p, mm.MM_F64)
    md = dev(wl.random_unit(n, seed=31), mm.MM_F64)
    with pytest.raises(mm.MMError) as e:
        mm.mm_llg_step(ctx, md, 0.0, 1e-13, mm.MM_RKF45, tol=1e-300)
    assert e.value.code == mm.MM_ERR_DT_UNDERFLOW
    md = dev(wl.random_unit(n, seed=31), mm.MM_F64)
    with pytest.raises(mm.MMError) as e:
        mm.mm_relax(ctx, md, t_max=1e-6, torque_tol=1e-12, max_steps=20)
    assert e.value.code == mm.MM_ERR_NOT_CONVERGED
    # the step cap is exact, rejected trials or not
    assert mm.mm_step_stats(ctx)[0] == 20
    t, dt, err = mm.mm_llg_step(ctx, md, 0.0, 1e-14, mm.MM_RKF45, tol=1e-5)   # still usable
    assert t > 0 and err <= 1e-5
    mm.mm_destroy(ctx)


EDGE_MESHES = [
    ((512, 1, 1), (1e-9, 2e-9, 3e-9)),     # the longest x line alone
    ((1, 512, 1), (2e-9, 1e-9, 3e-9)),     # the longest y line alone
    ((1, 1, 512), (2e-9, 3e-9, 1e-9)),     # the longest z line alone (Pz = 1024, generic z pass)
    ((8, 8, 512), (2e-9, 2e-9, 1e-9)),     # the largest nz on a small plane
    ((512, 4, 2), (1e-9, 1e-9, 1e-9)),     # the longest x pass with few rows
    ((3, 512, 2), (1e-9, 1e-9, 1e-9)),     # the longest y pass, a ragged x length
]


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("n,d", EDGE_MESHES)
def test_demag_at_the_size_limits(n, d, prec):
    """Meshes at the extents the library accepts (512 cells along an axis)
    and degenerate shapes (one cell thick in two directions): demag against
    the oracle's float64 convolution."""
    p = micromag.Problem(n, d)
    m = wl.random_unit(n, seed=13)
    ctx = gpu_ctx(p, prec)
    H = torch.empty(ctx.shape3, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    mm.mm_demag_field(ctx, dev(m, prec), H)
    assert rel_l2(host(H), p.demag_fft(m)) < TOL[prec]
    mm.mm_destroy(ctx)
