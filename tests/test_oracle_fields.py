"""Pins for the oracle's demag convolution (Eq. 4), exchange (Eq. 2),
anisotropy, Zeeman and energies against brute force, closed forms and the
energy-gradient identity."""

import numpy as np
import pytest

from oracle import micromag

MU0 = 4e-7 * np.pi


def unit_random(n, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    m = rng.normal(size=(3, nz, ny, nx))
    return m / np.linalg.norm(m, axis=0)


@pytest.mark.parametrize("n,d", [((4, 4, 2), (2.5e-9, 2.5e-9, 3e-9)),
                                 ((8, 8, 1), (2e-9, 2e-9, 2e-9)),
                                 ((5, 3, 3), (1e-9, 2e-9, 1.5e-9)),
                                 ((1, 1, 1), (1e-9, 1e-9, 1e-9)),
                                 ((1, 6, 1), (3e-9, 1e-9, 1e-9))])
def test_fft_convolution_equals_direct_sum(n, d):
    rng = np.random.default_rng(1)
    Ms = rng.uniform(2e5, 9e5, size=(n[2], n[1], n[0]))
    p = micromag.Problem(n, d, Ms_cell=Ms)
    m = unit_random(n, 3)
    a = p.demag_fft(m)
    b = p.demag_direct(m)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-13


def test_demag_is_self_adjoint():
    """N is symmetric (N_ij = N_ji) and even under r -> -r as an operator on the
    mesh, so <u, N v> = <N u, v> for any two fields (Ms = 1 here)."""
    n, d = (6, 5, 3), (2e-9, 3e-9, 1e-9)
    p = micromag.Problem(n, d, Ms=1.0)
    u, v = unit_random(n, 4), unit_random(n, 5)
    lhs = np.sum(u * p.demag_fft(v))
    rhs = np.sum(p.demag_fft(u) * v)
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=0)


def test_sampled_direct_sum_matches_full():
    n, d = (7, 4, 3), (2e-9, 2e-9, 2e-9)
    p = micromag.Problem(n, d)
    m = unit_random(n, 6)
    full = p.demag_fft(m)
    targets = [(0, 0, 0), (6, 3, 2), (3, 1, 1)]
    got = p.demag_direct(m, targets)
    for k, (x, y, z) in enumerate(targets):
        np.testing.assert_allclose(got[:, k], full[:, z, y, x], rtol=1e-12, atol=1e-9)


def test_exchange_uniform_is_zero():
    n, d = (6, 5, 3), (2.5e-9, 2.5e-9, 3e-9)
    p = micromag.Problem(n, d)
    m = np.zeros((3, 3, 5, 6))
    m[:] = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])[:, None, None, None]
    assert np.max(np.abs(p.exchange(m))) == 0.0


def test_exchange_spin_spiral_closed_form():
    nx, dx, A, Ms = 40, 2e-9, 1.3e-11, 8e5
    k = 2 * np.pi / (17 * dx)
    p = micromag.Problem((nx, 1, 1), (dx, 3e-9, 3e-9), Ms=Ms, A=A)
    x = np.arange(nx) * dx
    m = np.zeros((3, 1, 1, nx))
    m[0, 0, 0] = np.cos(k * x)
    m[1, 0, 0] = np.sin(k * x)
    H = p.exchange(m)
    pref = 2 * A / (MU0 * Ms * dx * dx)
    interior = slice(1, nx - 1)
    np.testing.assert_allclose(H[:, 0, 0, interior], pref * (2 * np.cos(k * dx) - 2) * m[:, 0, 0, interior],
                               rtol=1e-10, atol=1e-6)
    # free boundary: a single neighbour, H = pref (m_1 - m_0)
    np.testing.assert_allclose(H[:, 0, 0, 0], pref * (m[:, 0, 0, 1] - m[:, 0, 0, 0]), rtol=1e-12)
    np.testing.assert_allclose(H[:, 0, 0, -1], pref * (m[:, 0, 0, -2] - m[:, 0, 0, -1]), rtol=1e-12)


def _bond_energy(p, m):
    """Discrete exchange energy sum over bonds of V A_harm |m_i - m_j|^2 / d^2."""
    E = 0.0
    V = p.V
    for axis, h in ((2, p.d[0]), (1, p.d[1]), (0, p.d[2])):
        n = p.Ms.shape[axis]
        if n == 1:
            continue
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[axis], b[axis] = slice(0, n - 1), slice(1, n)
        a, b = tuple(a), tuple(b)
        Ai, Aj = p.A[a], p.A[b]
        Ah = 2 * Ai * Aj / (Ai + Aj)
        both = (p.Ms[a] > 0) & (p.Ms[b] > 0)
        dm2 = sum((m[c][a] - m[c][b]) ** 2 for c in range(3))
        E += np.sum(both * V * Ah * dm2 / (h * h))
    return E


def test_exchange_energy_equals_bond_sum_and_gradient():
    n, d = (5, 4, 3), (2e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(8)
    A = rng.uniform(0.5e-11, 2e-11, size=(3, 4, 5))
    Ms = rng.uniform(4e5, 9e5, size=(3, 4, 5))
    Ms[1, 2, 3] = 0.0  # a vacuum cell
    p = micromag.Problem(n, d, Ms_cell=Ms, A_cell=A)
    m = unit_random(n, 9)
    m[:, 1, 2, 3] = 0.0
    E = p.energies(m)[1]
    assert E == pytest.approx(_bond_energy(p, m), rel=1e-12, abs=0)
    # H_ex = -1/(mu0 Ms V) dE/dm for the bond energy (m not constrained)
    H = p.exchange(m)
    for (c, z, y, x) in [(0, 0, 0, 0), (2, 1, 1, 1), (1, 2, 3, 4), (0, 1, 3, 2)]:
        h = 1e-6
        mp_, mm_ = m.copy(), m.copy()
        mp_[c, z, y, x] += h
        mm_[c, z, y, x] -= h
        g = (_bond_energy(p, mp_) - _bond_energy(p, mm_)) / (2 * h)
        assert H[c, z, y, x] == pytest.approx(-g / (MU0 * Ms[z, y, x] * p.V), rel=1e-6, abs=0)
    assert np.all(H[:, 1, 2, 3] == 0.0)
    assert np.sum(Ms * np.sum(m * H, axis=0)) <= 0.0


def test_anisotropy_energy_limits():
    n, d = (4, 3, 2), (2e-9, 2e-9, 2e-9)
    p = micromag.Problem(n, d, Ku=5e5, u=(0, 0, 1))
    m = np.zeros((3, 2, 3, 4))
    m[2] = 1.0
    assert p.energies(m)[2] == pytest.approx(-5e5 * p.V * 24, rel=1e-14, abs=0)
    m2 = np.zeros_like(m)
    m2[0] = 1.0
    assert p.energies(m2)[2] == 0.0
    H = p.anisotropy(m)
    assert H[2, 0, 0, 0] == pytest.approx(2 * 5e5 / (MU0 * 8e5), rel=1e-14, abs=0)


def test_zeeman_energy():
    n, d = (3, 3, 1), (5e-9, 5e-9, 3e-9)
    h = np.array([-24.6e-3 / MU0, 4.3e-3 / MU0, 0.0])
    p = micromag.Problem(n, d, h_ext=h)
    m = np.zeros((3, 1, 3, 3))
    m[0] = 1.0
    assert p.energies(m)[3] == pytest.approx(-MU0 * 8e5 * p.V * 9 * h[0], rel=1e-14, abs=0)


def test_demag_energy_of_uniform_cube():
    """Uniform cube: E_demag = mu0/2 * Ms^2 * V_total / 3."""
    p = micromag.Problem((3, 3, 3), (2e-9, 2e-9, 2e-9))
    m = np.zeros((3, 3, 3, 3))
    m[1] = 1.0
    Vt = 27 * p.V
    assert p.energies(m)[0] == pytest.approx(0.5 * MU0 * 8e5 ** 2 * Vt / 3, rel=1e-12, abs=0)
