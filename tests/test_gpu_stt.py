"""Slonczewski spin-transfer torque through the C ABI against the oracle:
30 RK4 steps of a film with exchange, demag, anisotropy and the torque in
float64 and float32, the single-cell damping-like closed form, argument
checks and the adjoint's refusal."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

STT = dict(J=2e11, P=0.6, Lambda=1.5, eps_prime=0.1, p=(0.3, -0.4, 0.8))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def make(n, d, prec, alpha, stt, Ku=0.0):
    p = micromag.Problem(n, d, Ms=8e5, A=1.3e-11, alpha=alpha, Ku=Ku, u=(1, 0, 0), stt=stt)
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, alpha, Ku, (1, 0, 0))
    mm.mm_set_stt(ctx, stt["J"], stt["P"], stt["Lambda"], stt["eps_prime"], stt["p"], stt.get("d", 0.0))
    return p, ctx


@pytest.mark.parametrize("prec,tol", [(mm.MM_F64, 1e-11), (mm.MM_F32, 2e-5)], ids=["f64", "f32"])
def test_rk4_steps_match_oracle(prec, tol):
    n, d = (16, 16, 2), (2.5e-9, 2.5e-9, 2.5e-9)
    p, ctx = make(n, d, prec, 0.05, STT, Ku=2e5)
    m = wl.random_unit(n, seed=3)
    md = torch.tensor(m, dtype=torch.float64 if prec == mm.MM_F64 else torch.float32, device="cuda")
    for _ in range(30):
        mm.mm_llg_step(ctx, md, 0.0, 5e-14, mm.MM_RK4)
        m = p.rk4_step(m, 5e-14)
    assert np.linalg.norm(md.double().cpu().numpy() - m) / np.linalg.norm(m) < tol
    mm.mm_destroy(ctx)


def test_single_cell_damping_like_closed_form():
    d = (4e-9, 4e-9, 4e-9)
    alpha, eps_prime = 0.2, 0.15
    stt = dict(J=2e11, P=0.6, Lambda=1.0, eps_prime=eps_prime, p=(0, 0, 1))
    p, ctx = make((1, 1, 1), d, mm.MM_F64, alpha, stt)
    th0 = 2.0
    m = torch.tensor(np.array([np.sin(th0), 0.0, np.cos(th0)]).reshape(3, 1, 1, 1), dtype=torch.float64,
                     device="cuda")
    T, dt = 2e-10, 1e-12
    for _ in range(int(round(T / dt))):
        mm.mm_llg_step(ctx, m, 0.0, dt, mm.MM_RK4)
    beta = micromag.HBAR * 2e11 / (micromag.MU0 * micromag.QE * 8e5 * 4e-9)
    rate = micromag.GAMMA * beta * (0.3 + alpha * eps_prime) / (1 + alpha ** 2)
    th = float(torch.arccos(m[2, 0, 0, 0].clamp(-1, 1)))
    assert th == pytest.approx(2 * np.arctan(np.tan(th0 / 2) * np.exp(-rate * T)), rel=1e-8)
    mm.mm_destroy(ctx)


def test_arguments_and_adjoint_refusal():
    n, d = (8, 8, 1), (3e-9, 3e-9, 3e-9)
    ctx = mm.mm_init_mesh(*n, *d, precision=mm.MM_F64)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.1, 0.0, (0, 0, 1))
    with pytest.raises(mm.MMError):
        mm.mm_set_stt(ctx, 1e11, 0.5, 0.5, 0.0, (0, 0, 1))        # Lambda < 1
    with pytest.raises(mm.MMError):
        mm.mm_set_stt(ctx, 1e11, 0.5, 1.0, 0.0, (0, 0, 0))        # no polarisation
    mm.mm_set_stt(ctx, 1e11, 0.5, 1.0, 0.0, (0, 0, 2))
    m = torch.tensor(wl.random_unit(n, seed=1), dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(m)
    gMs = torch.zeros(ctx.shape1, dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MMError) as e:
        mm.mm_rk4_step_vjp(ctx, m, 1e-13, lam, gMs)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    mm.mm_set_stt(ctx, 0.0, 0.0, 1.0, 0.0, (0, 0, 1))            # off again
    mm.mm_rk4_step_vjp(ctx, m, 1e-13, lam, gMs)
    mm.mm_destroy(ctx)
