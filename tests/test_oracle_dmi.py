"""Pins for the oracle's DMI field (Eq. 3): closed forms for spin spirals
(interfacial cycloids along x and y, bulk helices along x and z), where the
central difference of a spiral of wave number q is exactly
-(sin(q d) / d) m, so H = -2 D sin(q d) / (mu0 Ms d) m in the interior; the
field against central finite differences of the independently written bond
energy; the -1/2 mu0 Ms V m.H energy equal to the bond energy; energy
conservation of RK4 at alpha = 0 with DMI."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

MU0 = 4e-7 * np.pi


def spiral(n, axis, q, d, kind):
    nx, ny, nz = n
    coords = [(np.arange(k) + 0.5) * h for k, h in zip(n, d)]
    s = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")[2 - axis]
    c, sn = np.cos(q * s), np.sin(q * s)
    z = np.zeros_like(s)
    if kind == "interfacial":
        return np.stack([sn, z, c]) if axis == 0 else np.stack([z, sn, c])
    return np.stack([z, c, sn]) if axis == 0 else np.stack([c, sn, z])


@pytest.mark.parametrize("kind,axis", [("interfacial", 0), ("interfacial", 1), ("bulk", 0), ("bulk", 2)])
def test_spiral_closed_form(kind, axis):
    n = [1, 1, 1]
    n[axis] = 24
    d = (2e-9, 3e-9, 2.5e-9)
    D, Ms = 3e-3, 8e5
    q = 2 * np.pi / (11 * d[axis])
    p = micromag.Problem(tuple(n), d, Ms=Ms, D=D, dmi=kind)
    m = spiral(tuple(n), axis, q, d, kind)
    H = p.dmi(m)
    ref = -2 * D * np.sin(q * d[axis]) / (MU0 * Ms * d[axis]) * m
    inner = [slice(None)] * 3
    inner[2 - axis] = slice(1, n[axis] - 1)
    inner = tuple(inner)
    for c in range(3):
        np.testing.assert_allclose(H[c][inner], ref[c][inner], rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("kind", ["interfacial", "bulk"])
def test_field_is_energy_gradient_with_vacuum_and_per_cell_ms(kind):
    n, d = (6, 5, 3), (2e-9, 2.5e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=1.5, seed=2)
    Ms[1, 2, 3] = 0.0
    p = micromag.Problem(n, d, Ms_cell=Ms, D=2e-3, dmi=kind)
    m = wl.random_unit(n, seed=3)
    H = p.dmi(m)
    h = 1e-6
    for c in range(3):
        for (z, y, x) in [(0, 0, 0), (1, 2, 2), (2, 4, 5), (1, 1, 3), (0, 3, 1)]:
            mp, mn = m.copy(), m.copy()
            mp[c, z, y, x] += h
            mn[c, z, y, x] -= h
            g = (p.dmi_bond_energy(mp) - p.dmi_bond_energy(mn)) / (2 * h)
            if Ms[z, y, x] == 0:
                assert H[c, z, y, x] == 0.0
                continue
            ref = -g / (MU0 * Ms[z, y, x] * p.V)
            assert H[c, z, y, x] == pytest.approx(ref, rel=1e-7, abs=1e-9 * np.abs(H).max())
    assert p.energies(m)[4] == pytest.approx(p.dmi_bond_energy(m), rel=1e-12, abs=0)


def test_rk4_conserves_energy_with_dmi_at_zero_damping():
    n, d = (8, 8, 2), (3e-9, 3e-9, 3e-9)
    p = micromag.Problem(n, d, Ms=8e5, A=1.3e-11, alpha=0.0, D=3e-3, dmi="interfacial")
    m = wl.smooth_unit(n, sigma_cells=2.0, seed=5)
    E0 = p.energies(m).sum()
    drift = []
    for dt in (4e-14, 2e-14):
        mm_ = m.copy()
        for _ in range(int(round(4e-12 / dt))):
            mm_ = p.rk4_step(mm_, dt)
        drift.append(abs(p.energies(mm_).sum() - E0) / abs(E0))
    assert drift[0] < 1e-6
    assert drift[1] < drift[0] / 10     # fourth-order drift
