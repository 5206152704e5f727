"""Gradients by their definition, CPU oracle (test infrastructure only).

The differentiation workload takes the per-cell saturation magnetisation Ms
as the design variable of a fixed-step RK4 LLG trajectory and the loss
L = (<m_z>(T) - target)^2, <.> the mean over magnetic cells.  The oracle's
gradient is the derivative itself, estimated per cell by central
differences with one Richardson step:
    D(h) = (L(Ms + h e_i) - L(Ms - h e_i)) / (2 h),
    dL/dMs_i ~ (4 D(h/2) - D(h)) / 3,          error O(h^4),
in float64 on the oracle's own trajectory (micromag.Problem.rk4_step).
"""

import numpy as np

from . import micromag


def mean_mz(p, m):
    mag = p.Ms > 0
    return float(np.sum(m[2] * mag) / np.sum(mag))


def trajectory(p, m0, dt, nsteps):
    m = m0.copy()
    for _ in range(nsteps):
        m = p.rk4_step(m, dt)
    return m


def loss(p, m0, dt, nsteps, target):
    return (mean_mz(p, trajectory(p, m0, dt, nsteps)) - target) ** 2


def richardson_central(f, x0, h):
    """(4 D(h/2) - D(h)) / 3 with D(h) = (f(x0 + h) - f(x0 - h)) / (2 h)."""
    d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
    d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


def grad_ms(p, m0, dt, nsteps, target, cells=None, rel_h=1e-3):
    """dL/dMs at the listed cells ((z, y, x) tuples; all cells if None)."""
    base = p.Ms.copy()
    if cells is None:
        cells = [tuple(c) for c in np.argwhere(base > 0)]
    out = []
    for c in cells:
        def f(v, c=c):
            p.Ms = base.copy()
            p.Ms[c] = v
            return loss(p, m0, dt, nsteps, target)
        out.append(richardson_central(f, base[c], rel_h * base[c]))
    p.Ms = base
    return np.array(out)


def energy_ms_gradient_fd(p, m, term, cells, rel_h=1e-3):
    """d E_term / d Ms_i by the same central-difference rule (term 0..3 of
    Problem.energies), for pinning this module against closed forms."""
    base = p.Ms.copy()
    out = []
    for c in cells:
        def f(v, c=c):
            p.Ms = base.copy()
            p.Ms[c] = v
            return p.energies(m)[term]
        out.append(richardson_central(f, base[c], rel_h * base[c]))
    p.Ms = base
    return np.array(out)
