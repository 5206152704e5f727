"""Pins for the oracle's LLG right-hand side (Eq. 1) and integrators: macrospin
closed form, |m| = 1, integrator order, energy conservation at alpha = 0 and
monotone decay at alpha > 0, the Fehlberg tableau's order conditions."""

import numpy as np
import pytest

from oracle import micromag

MU0 = micromag.MU0
GAMMA = micromag.GAMMA


def macrospin(alpha, H, theta0=1.0, phi0=0.3):
    """One cubic cell (its self-demag is parallel to m and exerts no torque),
    a field H along z."""
    p = micromag.Problem((1, 1, 1), (2e-9, 2e-9, 2e-9), alpha=alpha, h_ext=(0.0, 0.0, H))
    m = np.array([np.sin(theta0) * np.cos(phi0), np.sin(theta0) * np.sin(phi0), np.cos(theta0)]).reshape(3, 1, 1, 1)
    return p, m


def closed_form(alpha, H, t, theta0=1.0, phi0=0.3):
    g = GAMMA / (1 + alpha ** 2)
    theta = 2 * np.arctan(np.tan(theta0 / 2) * np.exp(-alpha * g * H * t))
    phi = phi0 + g * H * t
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


def test_macrospin_rk4_closed_form():
    alpha, H, dt, steps = 0.1, 1e5, 1e-13, 2000
    p, m = macrospin(alpha, H)
    for _ in range(steps):
        m = p.rk4_step(m, dt)
    ref = closed_form(alpha, H, dt * steps)
    np.testing.assert_allclose(m[:, 0, 0, 0], ref, atol=1e-9)
    assert np.linalg.norm(m[:, 0, 0, 0]) == pytest.approx(1.0, abs=1e-15)


def test_macrospin_rkf45_closed_form():
    alpha, H = 0.05, 2e5
    p, m = macrospin(alpha, H)
    t, dt, T = 0.0, 1e-14, 2e-10
    while t < T:
        dt = min(dt, T - t)
        m, t, dt, err, _ = micromag.rkf45_step(p, m, t, dt, 1e-7)
    np.testing.assert_allclose(m[:, 0, 0, 0], closed_form(alpha, H, t), atol=5e-6)


def test_rk4_global_order_four():
    alpha, H, T = 0.1, 1e5, 2e-10
    errs = []
    for dt in (2e-12, 1e-12):
        p, m = macrospin(alpha, H)
        for _ in range(int(round(T / dt))):
            m = p.rk4_step(m, dt)
        errs.append(np.linalg.norm(m[:, 0, 0, 0] - closed_form(alpha, H, T)))
    assert 12 < errs[0] / errs[1] < 20


def test_rkf45_local_orders():
    """One trial step from the same state: the 4th-order solution's local error
    scales as dt^5 and the embedded estimate |m5 - m4| as dt^5 too."""
    alpha, H = 0.1, 1e5
    out = []
    for dt in (4e-12, 2e-12):
        p, m = macrospin(alpha, H)
        k = []
        for s in range(6):
            ms = m.copy()
            for j in range(s):
                ms = ms + dt * micromag.FEHLBERG_A[s][j] * k[j]
            k.append(p.rhs(ms))
        m4 = m + dt * sum(micromag.FEHLBERG_B4[j] * k[j] for j in range(6))
        m5 = m + dt * sum(micromag.FEHLBERG_B5[j] * k[j] for j in range(6))
        # exact flow of the unnormalised ODE equals the closed form (|m| conserved)
        ref = closed_form(alpha, H, dt)
        out.append((np.linalg.norm(m4[:, 0, 0, 0] - ref), np.linalg.norm(m5[:, 0, 0, 0] - ref)))
    r4 = out[0][0] / out[1][0]
    r5 = out[0][1] / out[1][1]
    assert 26 < r4 < 38          # 2^5
    assert 52 < r5 < 80          # 2^6


def test_fehlberg_tableau_order_conditions():
    A = micromag.FEHLBERG_A
    c = np.array(micromag.FEHLBERG_C)
    b4 = np.array(micromag.FEHLBERG_B4)
    b5 = np.array(micromag.FEHLBERG_B5)
    for s in range(6):
        assert sum(A[s]) == pytest.approx(c[s], abs=1e-15)
    Am = np.zeros((6, 6))
    for s in range(6):
        Am[s, :s] = A[s]
    for b, order in ((b4, 4), (b5, 5)):
        assert b.sum() == pytest.approx(1, abs=1e-14)
        assert b @ c == pytest.approx(1 / 2, abs=1e-14)
        assert b @ c ** 2 == pytest.approx(1 / 3, abs=1e-14)
        assert b @ Am @ c == pytest.approx(1 / 6, abs=1e-14)
        assert b @ c ** 3 == pytest.approx(1 / 4, abs=1e-14)
        assert b @ (c * (Am @ c)) == pytest.approx(1 / 8, abs=1e-14)
        assert b @ Am @ c ** 2 == pytest.approx(1 / 12, abs=1e-14)
        assert b @ Am @ Am @ c == pytest.approx(1 / 24, abs=1e-14)
    assert b5 @ c ** 4 == pytest.approx(1 / 5, abs=1e-14)
    assert b5 @ Am @ Am @ Am @ c == pytest.approx(1 / 120, abs=1e-14)


def _film(alpha):
    n, d = (8, 8, 2), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d, alpha=alpha, Ku=1e5, u=(0.0, 0.6, 0.8), h_ext=(1e4, 0.0, -2e4))
    rng = np.random.default_rng(11)
    m = rng.normal(size=(3, 2, 8, 8)) * 0.3
    m[2] += 1.0
    m /= np.linalg.norm(m, axis=0)
    return p, m


def test_energy_conserved_at_zero_damping_with_dt4_drift():
    drifts = []
    for dt in (2e-14, 1e-14):
        p, m = _film(0.0)
        E0 = p.energies(m).sum()
        for _ in range(int(round(4e-13 / dt))):
            m = p.rk4_step(m, dt)
        drifts.append(abs(p.energies(m).sum() - E0) / abs(E0))
    assert drifts[1] < 1e-6
    assert drifts[0] / drifts[1] > 8


def test_energy_decays_monotonically_with_damping():
    p, m = _film(0.5)
    E = [p.energies(m).sum()]
    for _ in range(30):
        m = p.rk4_step(m, 2e-14)
        E.append(p.energies(m).sum())
        assert np.max(np.abs(np.linalg.norm(m, axis=0) - 1)) < 1e-14
    assert all(e1 < e0 for e0, e1 in zip(E, E[1:]))


def test_relax_macrospin_aligns_with_field():
    p, m = macrospin(0.5, 3e5)
    m, t, steps = micromag.relax(p, m, t_max=5e-9, torque_tol=1e-4, max_steps=100000)
    assert t < 5e-9                      # stopped on the torque criterion
    assert p.max_torque(m) <= 1e-4
    assert m[2, 0, 0, 0] > 1 - 1e-7


def test_rkf45_rejects_and_recovers():
    p, m = _film(0.02)
    m1, t1, dt1, err, rejected = micromag.rkf45_step(p, m, 0.0, 1e-11, 1e-5)
    assert rejected >= 1 and err <= 1e-5 and t1 < 1e-11
