"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

Holds none of the method's arithmetic: only magnetisation and material
patterns, drawn from numpy's PCG64 with fixed seeds.  Arrays are float64,
vectors laid out [3][nz][ny][nx] (x fastest), scalars [nz][ny][nx].

Workloads (mesh, cell size, material) are the configurations the library is
measured and checked on:
  film64     64 x 64 x 4,  2.5 x 2.5 x 3 nm, permalloy, random m (fixed-step RK4)
  film512    512 x 512 x 16, 2 nm cubes, permalloy alpha 0.5, vortex + 5 % noise (RKF45)
  cube256    256^3, 1 nm cubes, Ku 5e5 along z, random m
  design256  256 x 256 x 4, 3 nm cubes, smooth per-cell Ms in [4e5, 9e5]
  film256    256 x 256 x 1, 4 nm cubes, permalloy
"""

import numpy as np

WORKLOADS = {
    "film64": dict(n=(64, 64, 4), d=(2.5e-9, 2.5e-9, 3e-9), Ms=8.0e5, A=1.3e-11, alpha=0.02, Ku=0.0),
    "film512": dict(n=(512, 512, 16), d=(2e-9, 2e-9, 2e-9), Ms=8.0e5, A=1.3e-11, alpha=0.5, Ku=0.0),
    "cube256": dict(n=(256, 256, 256), d=(1e-9, 1e-9, 1e-9), Ms=8.0e5, A=1.3e-11, alpha=0.02, Ku=5e5),
    "design256": dict(n=(256, 256, 4), d=(3e-9, 3e-9, 3e-9), Ms=8.0e5, A=1.3e-11, alpha=0.02, Ku=0.0),
    "film256": dict(n=(256, 256, 1), d=(4e-9, 4e-9, 4e-9), Ms=8.0e5, A=1.3e-11, alpha=0.5, Ku=0.0),
}


def _unit(v):
    nrm = np.sqrt(np.sum(v * v, axis=0))
    return v / np.where(nrm > 0, nrm, 1.0)


def random_unit(n, seed):
    """Independent uniformly random unit vectors (normalised N(0, I3) draws)."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    return _unit(rng.standard_normal((3, nz, ny, nx)))


def uniform(n, direction=(0.0, 0.0, 1.0)):
    nx, ny, nz = n
    v = np.asarray(direction, dtype=np.float64)
    v = v / np.linalg.norm(v)
    return np.broadcast_to(v[:, None, None, None], (3, nz, ny, nx)).copy()


def vortex(n, d, core_radius=10e-9, noise=0.05, seed=1, chirality=1.0, polarity=1.0, center=(0.0, 0.0)):
    """Vortex at ``center`` (m, from the mesh centre): m_z = p exp(-r^2 / rc^2),
    in-plane c (-sin phi, cos phi) sqrt(1 - m_z^2), plus ``noise`` N(0, I3),
    renormalised."""
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) * d[0] - nx * d[0] / 2 - center[0]
    y = (np.arange(ny) + 0.5) * d[1] - ny * d[1] / 2 - center[1]
    Y, X = np.meshgrid(y, x, indexing="ij")
    r2 = X * X + Y * Y
    phi = np.arctan2(Y, X)
    mz = polarity * np.exp(-r2 / core_radius ** 2)
    ip = np.sqrt(np.clip(1 - mz * mz, 0, None))
    m = np.stack([-chirality * np.sin(phi) * ip, chirality * np.cos(phi) * ip, mz])
    m = np.broadcast_to(m[:, None], (3, nz, ny, nx)).copy()
    if noise:
        rng = np.random.default_rng(seed)
        m = m + noise * rng.standard_normal(m.shape)
    return _unit(m)


def domain_wall(n, d, width=20e-9, axis=0, seed=None, noise=0.0, offset=0.0):
    """Neel-type wall across ``axis`` at ``offset`` (m) from the middle:
    m_z = -tanh(s / w)."""
    nx, ny, nz = n
    coords = [(np.arange(k) + 0.5) * h - k * h / 2 for k, h in zip(n, d)]
    s = coords[axis] - offset
    mz = -np.tanh(s / width)
    mt = np.sqrt(1 - mz * mz)
    shape = [1, 1, 1]
    shape[2 - axis] = n[axis]
    mz = mz.reshape(shape)
    mt = mt.reshape(shape)
    m = np.zeros((3, nz, ny, nx))
    m[axis] = np.broadcast_to(mt, (nz, ny, nx))
    m[2] = np.broadcast_to(mz, (nz, ny, nx))
    if axis == 2:
        m[0] = np.broadcast_to(mt, (nz, ny, nx))
        m[2] = np.broadcast_to(mz, (nz, ny, nx))
    if noise:
        rng = np.random.default_rng(seed)
        m = m + noise * rng.standard_normal(m.shape)
    return _unit(m)


def smooth_field(n, lo, hi, sigma_cells=8.0, seed=3):
    """Gaussian-filtered N(0, 1) (sigma in cells, periodic), min-max rescaled to [lo, hi]."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((nz, ny, nx))
    k = [np.fft.fftfreq(v) for v in (nz, ny, nx)]
    KZ, KY, KX = np.meshgrid(*k, indexing="ij")
    g = np.exp(-2 * (np.pi * sigma_cells) ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    s = np.real(np.fft.ifftn(np.fft.fftn(w) * g))
    s = (s - s.min()) / (s.max() - s.min())
    return lo + (hi - lo) * s


def smooth_unit(n, sigma_cells=4.0, seed=0):
    """Unit vectors from three Gaussian-filtered N(0, 1) fields (periodic),
    normalised: a random texture with correlation length ~sigma cells."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, nz, ny, nx))
    k = [np.fft.fftfreq(m) for m in (nz, ny, nx)]
    KZ, KY, KX = np.meshgrid(*k, indexing="ij")
    g = np.exp(-2 * (np.pi * sigma_cells) ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    v = np.real(np.fft.ifftn(np.fft.fftn(v, axes=(1, 2, 3)) * g, axes=(1, 2, 3)))
    return _unit(v)


def film_state(n, d, seed):
    """One of four film textures, chosen and shaped by ``seed``: random unit
    vectors, a vortex (random centre, chirality, polarity, core), a domain
    wall (random axis, position, width) or a smooth random texture."""
    rng = np.random.default_rng(seed)
    kind = seed % 4
    Lx, Ly = n[0] * d[0], n[1] * d[1]
    if kind == 0:
        return random_unit(n, seed=seed)
    if kind == 1:
        return vortex(n, d, core_radius=rng.uniform(5e-9, 20e-9), noise=rng.uniform(0.0, 0.2), seed=seed,
                      chirality=rng.choice([-1.0, 1.0]), polarity=rng.choice([-1.0, 1.0]),
                      center=(rng.uniform(-0.25, 0.25) * Lx, rng.uniform(-0.25, 0.25) * Ly))
    if kind == 2:
        axis = int(rng.integers(0, 2))
        return domain_wall(n, d, width=rng.uniform(5e-9, 30e-9), axis=axis, seed=seed, noise=rng.uniform(0.0, 0.2),
                           offset=rng.uniform(-0.3, 0.3) * (Lx if axis == 0 else Ly))
    return smooth_unit(n, sigma_cells=rng.uniform(2.0, 12.0), seed=seed)
