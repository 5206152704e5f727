"""Pins for the oracle's finite-difference gradients against closed forms:
E_demag = -(mu0/2) V sum Ms m.H_d is quadratic in Ms with the symmetric
Newell operator, so dE_demag/dMs_k = -mu0 V m_k.H_d,k; E_zee = -mu0 V sum
Ms m.H_ext gives dE_zee/dMs_k = -mu0 V m_k.H_ext; and a single cubic cell's
self-demag field is parallel to m, so its trajectory does not depend on Ms."""

import numpy as np
import pytest

import workloads as wl
from oracle import adjoint, micromag

MU0 = micromag.MU0


def test_fd_gradient_of_demag_energy_closed_form():
    n, d = (6, 5, 2), (2e-9, 2e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=1.5, seed=3)
    p = micromag.Problem(n, d, Ms_cell=Ms)
    m = wl.random_unit(n, seed=4)
    cells = [(0, 0, 0), (1, 4, 5), (0, 2, 3), (1, 1, 1)]
    fd = adjoint.energy_ms_gradient_fd(p, m, 0, cells)
    H = p.demag_fft(m)
    closed = np.array([-MU0 * p.V * np.dot(m[:, z, y, x], H[:, z, y, x]) for (z, y, x) in cells])
    np.testing.assert_allclose(fd, closed, rtol=1e-9)


def test_fd_gradient_of_zeeman_energy_closed_form():
    n, d = (4, 4, 1), (5e-9, 5e-9, 3e-9)
    h = np.array([1e4, -2e4, 3e4])
    p = micromag.Problem(n, d, h_ext=h)
    m = wl.random_unit(n, seed=5)
    cells = [(0, 0, 0), (0, 3, 2)]
    fd = adjoint.energy_ms_gradient_fd(p, m, 3, cells)
    closed = np.array([-MU0 * p.V * np.dot(m[:, z, y, x], h) for (z, y, x) in cells])
    np.testing.assert_allclose(fd, closed, rtol=1e-10)


def test_single_cube_trajectory_does_not_depend_on_ms():
    p = micromag.Problem((1, 1, 1), (2e-9, 2e-9, 2e-9), alpha=0.1, h_ext=(0.0, 0.0, 1e5))
    m0 = wl.random_unit((1, 1, 1), seed=6)
    g = adjoint.grad_ms(p, m0, 1e-13, 20, 0.3)
    assert abs(g[0]) < 1e-12


def test_richardson_is_fourth_order():
    f = lambda x: np.sin(3 * x) * np.exp(x)
    exact = lambda x: (3 * np.cos(3 * x) + np.sin(3 * x)) * np.exp(x)
    e1 = abs(adjoint.richardson_central(f, 0.4, 0.1) - exact(0.4))
    e2 = abs(adjoint.richardson_central(f, 0.4, 0.05) - exact(0.4))
    assert 10 < e1 / e2 < 22
