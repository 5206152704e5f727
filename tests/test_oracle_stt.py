"""Pins for the oracle's Slonczewski torque: the right-hand side equals the
solution of the implicit Gilbert form dm/dt = X + alpha m x dm/dt (X the
precession and spin-torque terms) found by a linear solve per cell; with
Lambda = 1 (constant eps) and no field the polar angle from p follows
tan(theta/2) = tan(theta0/2) exp(-gamma beta (eps + alpha eps') t / (1 + alpha^2))
and the pure field-like term precesses m about p at gamma beta eps' / (1 + alpha^2)."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

MU0, GAMMA = micromag.MU0, micromag.GAMMA


def stt(**kw):
    base = dict(J=2e11, P=0.6, Lambda=1.5, eps_prime=0.1, p=(0.3, -0.4, 0.8))
    base.update(kw)
    return base


def test_rhs_solves_the_gilbert_form():
    n, d = (6, 4, 2), (3e-9, 3e-9, 2e-9)
    a = 0.37
    p = micromag.Problem(n, d, Ms=7e5, A=1.1e-11, alpha=a, Ku=1e5, u=(1, 1, 0), stt=stt())
    m = wl.random_unit(n, seed=2)
    H = p.h_eff(m)
    got = p.llg_rhs(m, H)
    st = p.stt
    pv = st["p"]
    beta = micromag.HBAR * st["J"] / (MU0 * micromag.QE * 7e5 * st["d"])
    L2 = st["Lambda"] ** 2
    for idx in [(0, 0, 0), (1, 3, 5), (0, 2, 1)]:
        mi = m[(slice(None),) + idx]
        Hi = H[(slice(None),) + idx]
        eps = st["P"] * L2 / ((L2 + 1) + (L2 - 1) * mi @ pv)
        X = -GAMMA * np.cross(mi, Hi) + GAMMA * beta * (eps * np.cross(mi, np.cross(pv, mi)) + st["eps_prime"] * np.cross(pv, mi))
        # (I - alpha [m]_x) v = X
        mx = np.array([[0, -mi[2], mi[1]], [mi[2], 0, -mi[0]], [-mi[1], mi[0], 0]])
        v = np.linalg.solve(np.eye(3) - a * mx, X)
        np.testing.assert_allclose(got[(slice(None),) + idx], v, rtol=1e-12, atol=1e-12 * np.abs(v).max())


@pytest.mark.parametrize("alpha,eps_prime", [(0.0, 0.0), (0.2, 0.0), (0.2, 0.15)])
def test_damping_like_relaxation_closed_form(alpha, eps_prime):
    # one cubic cell: isotropic self demag, no exchange, no field
    d = (4e-9, 4e-9, 4e-9)
    pv = np.array([0.0, 0.0, 1.0])
    p = micromag.Problem((1, 1, 1), d, Ms=8e5, alpha=alpha, stt=stt(Lambda=1.0, eps_prime=eps_prime, p=pv))
    th0 = 2.0
    m = np.array([np.sin(th0), 0.0, np.cos(th0)]).reshape(3, 1, 1, 1)
    beta = micromag.HBAR * 2e11 / (MU0 * micromag.QE * 8e5 * 4e-9)
    eps = 0.6 / 2
    rate = GAMMA * beta * (eps + alpha * eps_prime) / (1 + alpha ** 2)
    dt, T = 1e-12, 2e-10
    for _ in range(int(round(T / dt))):
        m = p.rk4_step(m, dt)
    th = np.arccos(np.clip(m[2, 0, 0, 0], -1, 1))
    ref = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-rate * T))
    assert th == pytest.approx(ref, rel=1e-8, abs=0)


def test_field_like_precession_closed_form():
    d = (4e-9, 4e-9, 4e-9)
    p = micromag.Problem((1, 1, 1), d, Ms=8e5, alpha=0.0, stt=stt(P=0.0, Lambda=1.0, eps_prime=0.3, p=(0, 0, 1)))
    th0, T, dt = 1.0, 1e-10, 1e-13
    m = np.array([np.sin(th0), 0.0, np.cos(th0)]).reshape(3, 1, 1, 1)
    for _ in range(int(round(T / dt))):
        m = p.rk4_step(m, dt)
    beta = micromag.HBAR * 2e11 / (MU0 * micromag.QE * 8e5 * 4e-9)
    w = GAMMA * beta * 0.3
    phi = np.arctan2(m[1, 0, 0, 0], m[0, 0, 0, 0])
    # p x m = rotation of m about +p: phi grows at rate w
    assert phi == pytest.approx(w * T, abs=1e-9)
    assert m[2, 0, 0, 0] == pytest.approx(np.cos(th0), abs=1e-12)
