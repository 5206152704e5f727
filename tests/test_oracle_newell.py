"""Pins for the oracle's Newell tensor (Eq. 4's kernel N) against what the
mathematics fixes: the cube self term, the trace identity, Aharoni's closed-form
prism factors, the dipole limit, and a 60-digit evaluation of the exact formula
that bounds both the extended-precision near field and the far-field series."""

import math

import mpmath as mp
import numpy as np
import pytest

from oracle import micromag, newell

COMPS = newell.COMPONENTS


def aharoni_Dz(a, b, c):
    """Aharoni, J. Appl. Phys. 83, 3432 (1998): D_z of a 2a x 2b x 2c prism."""
    r = math.sqrt(a * a + b * b + c * c)
    rab, rbc, rac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    s = ((b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
         + b / (2 * c) * math.log((rab + a) / (rab - a))
         + a / (2 * c) * math.log((rab + b) / (rab - b))
         + c / (2 * a) * math.log((rbc - b) / (rbc + b))
         + c / (2 * b) * math.log((rac - a) / (rac + a))
         + 2 * math.atan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (rac + rbc)
         - (rab ** 3 + rbc ** 3 + rac ** 3) / (3 * a * b * c))
    return s / math.pi


def test_cube_self_term():
    d = (1e-9, 1e-9, 1e-9)
    for c in ("xx", "yy", "zz"):
        assert newell.newell_exact(c, 0, 0, 0, d) == pytest.approx(1 / 3, abs=1e-15)
    for c in ("xy", "xz", "yz"):
        assert newell.newell_exact(c, 0, 0, 0, d) == 0.0


@pytest.mark.parametrize("d", [(2.5e-9, 2.5e-9, 3e-9), (4e-9, 4e-9, 0.7e-9), (1e-9, 3e-9, 2e-9)])
def test_trace_self_and_offsets(d):
    tr0 = sum(newell.newell_exact(c, 0, 0, 0, d) for c in ("xx", "yy", "zz"))
    assert tr0 == pytest.approx(1.0, abs=1e-15)
    rng = np.random.default_rng(7)
    I, J, K = rng.integers(-12, 13, size=(3, 40))
    keep = (I != 0) | (J != 0) | (K != 0)
    I, J, K = I[keep], J[keep], K[keep]
    tr = sum(newell.newell_tensor(c, I, J, K, d) for c in ("xx", "yy", "zz"))
    scale = np.abs(newell.newell_tensor("xx", I, J, K, d)) + 1e-30
    assert np.max(np.abs(tr)) < 1e-14
    assert np.max(np.abs(tr) / scale) < 1e-6


@pytest.mark.parametrize("abc", [(1.0, 1.0, 1.0), (1.0, 2.0, 0.5), (3.0, 1.0, 0.2), (10.0, 10.0, 0.1)])
def test_prism_self_term_equals_aharoni(abc):
    a, b, c = abc
    got = newell.newell_exact("zz", 0, 0, 0, (2 * a, 2 * b, 2 * c))
    assert got == pytest.approx(aharoni_Dz(a, b, c), rel=1e-12, abs=0)
    # cycled axes: D_x of the prism is D_z of the prism with axes cycled
    gotx = newell.newell_exact("xx", 0, 0, 0, (2 * a, 2 * b, 2 * c))
    assert gotx == pytest.approx(aharoni_Dz(b, c, a), rel=1e-12, abs=0)


@pytest.mark.parametrize("n,d", [((6, 5, 3), (2.5e-9, 2.5e-9, 3e-9)),
                                 ((8, 8, 2), (2e-9, 2e-9, 2e-9)),
                                 ((7, 3, 1), (1e-9, 2e-9, 0.5e-9))])
def test_body_average_equals_prism_factor(n, d):
    """Newell is the exact cell-averaged tensor, so the average over all cell
    pairs of an n-cell prism is the demag factor of the whole prism."""
    p = micromag.Problem(n, d)
    nx, ny, nz = n
    big = (nx * d[0], ny * d[1], nz * d[2])
    for c, name in ((0, "xx"), (1, "yy"), (2, "zz")):
        m = np.zeros((3, nz, ny, nx))
        m[c] = 1.0
        H = p.demag_direct(m)
        avg = -np.mean(H[c]) / p.Ms[0, 0, 0]
        assert avg == pytest.approx(newell.newell_exact(name, 0, 0, 0, big), abs=1e-13)
    # thin film limit N_zz -> 1: 1 - D_z shrinks as the aspect ratio grows
    gaps = [1 - newell.newell_exact("zz", 0, 0, 0, (2 * a, 2 * a, 1.0)) for a in (10.0, 100.0, 1000.0, 10000.0)]
    assert all(g1 < g0 for g0, g1 in zip(gaps, gaps[1:]))
    assert gaps[-1] < 5e-4


def test_uniform_cube_field_is_minus_ms_over_three():
    p = micromag.Problem((4, 4, 4), (1e-9, 1e-9, 1e-9))
    m = np.zeros((3, 4, 4, 4))
    m[2] = 1.0
    H = p.demag_fft(m)
    assert np.mean(H[2]) == pytest.approx(-p.Ms[0, 0, 0] / 3, rel=1e-13, abs=0)
    assert np.max(np.abs(np.mean(H[:2], axis=(1, 2, 3)))) < 1e-9 * p.Ms[0, 0, 0]


def dipole(comp, I, J, K, d):
    x, y, z = I * d[0], J * d[1], K * d[2]
    r = math.sqrt(x * x + y * y + z * z)
    v = {"x": x, "y": y, "z": z}
    delta = 1.0 if comp[0] == comp[1] else 0.0
    return d[0] * d[1] * d[2] / (4 * math.pi) * (delta * r * r - 3 * v[comp[0]] * v[comp[1]]) / r ** 5


def test_far_field_tends_to_dipole():
    d = (2.5e-9, 2.5e-9, 3e-9)
    prev = None
    for s in (4, 8, 16, 32):
        errs = []
        for c in COMPS:
            I, J, K = 3 * s, 2 * s, s
            ex = float(newell.newell_exact(c, I, J, K, d))
            errs.append(abs(ex - dipole(c, I, J, K, d)) / abs(dipole("xx", I, J, K, d)))
        e = max(errs)
        if prev is not None:
            # leading correction is O((d/R)^2): doubling R divides it by about 4
            assert 2.5 < prev / e < 6.0
        prev = e
    assert prev < 1e-3


# ---- 60-digit reference evaluation of the exact formula -------------------------

def _f_mp(x, y, z):
    x, y, z = abs(x), abs(y), abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = mp.sqrt(x2 + y2 + z2)
    r = (2 * x2 - y2 - z2) * R / 6
    if x2 + z2 > 0:
        r += y / 2 * (z2 - x2) * mp.asinh(y / mp.sqrt(x2 + z2))
    if x2 + y2 > 0:
        r += z / 2 * (y2 - x2) * mp.asinh(z / mp.sqrt(x2 + y2))
    if x * R > 0:
        r -= x * y * z * mp.atan(y * z / (x * R))
    return r


def _g_mp(x, y, z):
    s = mp.sign(x) * mp.sign(y)
    x, y, z = abs(x), abs(y), abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = mp.sqrt(x2 + y2 + z2)
    r = -x * y * R / 3
    if x2 + y2 > 0:
        r += x * y * z * mp.asinh(z / mp.sqrt(x2 + y2))
    if y2 + z2 > 0:
        r += y / 6 * (3 * z2 - y2) * mp.asinh(x / mp.sqrt(y2 + z2))
    if x2 + z2 > 0:
        r += x / 6 * (3 * z2 - x2) * mp.asinh(y / mp.sqrt(x2 + z2))
    if z * R > 0:
        r -= z * z2 / 6 * mp.atan(x * y / (z * R))
    if y * R > 0:
        r -= z * y2 / 2 * mp.atan(x * z / (y * R))
    if x * R > 0:
        r -= z * x2 / 2 * mp.atan(y * z / (x * R))
    return s * r


_PERM = {"xx": (_f_mp, (0, 1, 2)), "yy": (_f_mp, (1, 2, 0)), "zz": (_f_mp, (2, 0, 1)),
         "xy": (_g_mp, (0, 1, 2)), "xz": (_g_mp, (0, 2, 1)), "yz": (_g_mp, (1, 2, 0))}


def newell_mp(comp, I, J, K, d):
    with mp.workdps(60):
        dx, dy, dz = (mp.mpf(v) for v in d)
        fn, perm = _PERM[comp]
        acc = mp.mpf(0)
        for ex in (-1, 0, 1):
            for ey in (-1, 0, 1):
                for ez in (-1, 0, 1):
                    w = (2 if ex == 0 else -1) * (2 if ey == 0 else -1) * (2 if ez == 0 else -1)
                    p = ((I + ex) * dx, (J + ey) * dy, (K + ez) * dz)
                    acc += w * fn(p[perm[0]], p[perm[1]], p[perm[2]])
        return acc / (4 * mp.pi * dx * dy * dz)


@pytest.mark.parametrize("d", [(2.5e-9, 2.5e-9, 3e-9), (4e-9, 4e-9, 0.7e-9)])
def test_near_field_extended_precision_matches_60_digits(d):
    offs = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, -1, 1), (3, -2, 1), (-7, 5, 2), (9, 0, -3)]
    for c in COMPS:
        for (I, J, K) in offs:
            ref = float(newell_mp(c, I, J, K, d))
            got = float(newell.newell_exact(c, I, J, K, d))
            assert abs(got - ref) < 2e-16, (c, I, J, K, got, ref)


@pytest.mark.parametrize("d", [(2.5e-9, 2.5e-9, 3e-9), (1e-9, 1e-9, 1e-9), (4e-9, 4e-9, 0.7e-9)])
def test_series_truncation_below_1e17_at_switch_radius(d):
    """At the near/far switch (16 largest edges) the K = 4 series must equal
    the exact element to far below FP64 roundoff of the near elements."""
    dmax = max(d)
    offs = []
    for direction in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (2, -1, 3), (-3, 2, 1)]:
        v = np.array([direction[0] * 1.0, direction[1] * 1.0, direction[2] * 1.0])
        phys = v * np.array(d)
        scale = newell.NEAR_CELLS * dmax / np.linalg.norm(phys) * 1.02
        I, J, K = (int(math.ceil(abs(t) * scale)) * int(np.sign(t)) for t in v)
        offs.append((I, J, K))
    for c in COMPS:
        for (I, J, K) in offs:
            assert not newell.is_near(I, J, K, d)
            ref = float(newell_mp(c, I, J, K, d))
            got = float(newell.newell_series(c, I, J, K, d))
            assert abs(got - ref) < 1e-17, (c, I, J, K, got, ref)


def test_inverse_r_derivatives_match_numerical_differentiation():
    x, y, z = 1.3, -0.7, 2.1
    der = newell.inverse_r_derivatives(np.array(x), np.array(y), np.array(z), 6)
    g = lambda a, b, c: 1 / mp.sqrt(a * a + b * b + c * c)
    with mp.workdps(40):
        for key in [(0, 0, 0), (1, 0, 0), (2, 0, 0), (1, 1, 0), (2, 2, 2), (3, 1, 2), (0, 4, 2), (6, 0, 0)]:
            ref = float(mp.diff(g, (mp.mpf(x), mp.mpf(y), mp.mpf(z)), key))
            assert float(der[key]) == pytest.approx(ref, rel=1e-11, abs=1e-13)


def test_symmetries():
    d = (2.5e-9, 2.5e-9, 3e-9)
    I, J, K = 5, 3, 2
    for c in COMPS:
        v = newell.newell_tensor(c, I, J, K, d)
        par = {"xx": (1, 1, 1), "yy": (1, 1, 1), "zz": (1, 1, 1),
               "xy": (-1, -1, 1), "xz": (-1, 1, -1), "yz": (1, -1, -1)}[c]
        assert newell.newell_tensor(c, -I, J, K, d) == pytest.approx(par[0] * v, rel=1e-13, abs=1e-22)
        assert newell.newell_tensor(c, I, -J, K, d) == pytest.approx(par[1] * v, rel=1e-13, abs=1e-22)
        assert newell.newell_tensor(c, I, J, -K, d) == pytest.approx(par[2] * v, rel=1e-13, abs=1e-22)
    # the cubic-cell tensor is invariant under exchanging x and y roles
    dc = (1e-9, 1e-9, 1e-9)
    assert newell.newell_tensor("xx", 4, 2, 1, dc) == pytest.approx(newell.newell_tensor("yy", 2, 4, 1, dc), rel=1e-12, abs=0)
    assert newell.newell_tensor("xz", 4, 2, 1, dc) == pytest.approx(newell.newell_tensor("yz", 2, 4, 1, dc), rel=1e-12, abs=0)
