"""Newell demagnetisation tensor, CPU oracle (test infrastructure only).

The paper computes the demag field (Eq. 4) as a discrete convolution with a
kernel N "computed using Newell's formula".  The formulas themselves are not
printed; this module restates them from Newell, Williams & Dunlop (1993):

    N_ij(R) = -(1/V) * integral over cell A, integral over cell B of
              d_i d_j G(R + u - v) du dv,     G(r) = 1 / (4 pi |r|),

the field of a uniformly magnetised cuboid averaged over another one, with
H = -N M.  Newell's auxiliary functions f (diagonal) and g (off-diagonal) are
sixth antiderivatives of that integrand, and the tensor element is the
27-point product of second differences of f (or g) with weights (-1, 2, -1)
per axis, divided by 4 pi V.

Two evaluations, used by distance:

* near field (|R| < NEAR_CELLS * max cell edge): the exact formula.  The
  27-point sum cancels about R^6 units of roundoff, so it runs in numpy
  ``longdouble`` (80-bit on x86-64, IEEE binary128 on aarch64).
* far field: the Taylor expansion of the cell-averaged integrand.  u - v has
  the triangular ("tent") distribution on [-d, d] per axis, whose even moments
  give E[w^(2a)] / (2a)! = 2 d^(2a) / (2a + 2)!, so

      N_ij(R) = -(V / 4 pi) * sum_{a+b+c <= K} C_a(dx) C_b(dy) C_c(dz)
                 * d_x^(2a) d_y^(2b) d_z^(2c) d_i d_j (1/r) at R,

  C_a(d) = 2 d^(2a) / (2a+2)!.  The Cartesian derivatives of 1/r come from the
  McMurchie-Davidson recurrence (J. Comput. Phys. 26, 218 (1978)).  With
  K = 4 and |R| >= 16 max-edges the truncation error is below 1e-17 in
  absolute value (pinned against a 60-digit evaluation of the exact formula in
  the tests), far below FP64 roundoff of the near elements.

Everything here is float64 except the exact near field.
"""

import math
from functools import lru_cache

import numpy as np

NEAR_CELLS = 16.0     # switch radius in units of the largest cell edge
SERIES_ORDER = 4      # K: total order a+b+c of the tent-moment series
LD = np.longdouble

# component order used throughout: xx, yy, zz, xy, xz, yz
COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")


def newell_f(x, y, z):
    """Newell's f(x, y, z) for N_xx; even in every argument, symmetric in y, z.

    Terms whose prefactor vanishes are taken as 0 (their limits)."""
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = (2 * x2 - y2 - z2) * R / 6
    with np.errstate(divide="ignore", invalid="ignore"):
        rxz = np.sqrt(x2 + z2)
        rxy = np.sqrt(x2 + y2)
        t1 = y / 2 * (z2 - x2) * np.arcsinh(y / rxz)
        t2 = z / 2 * (y2 - x2) * np.arcsinh(z / rxy)
        t3 = x * y * z * np.arctan(y * z / (x * R))
    out = out + np.where(rxz > 0, t1, 0) + np.where(rxy > 0, t2, 0)
    out = out - np.where(x * R > 0, t3, 0)
    return out


def newell_g(x, y, z):
    """Newell's g(x, y, z) for N_xy; odd in x and y, even in z, symmetric in x, y.

    Evaluated at |x|, |y|, |z| and given the sign sign(x) sign(y)."""
    sgn = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = -x * y * R / 3
    with np.errstate(divide="ignore", invalid="ignore"):
        rxy = np.sqrt(x2 + y2)
        ryz = np.sqrt(y2 + z2)
        rxz = np.sqrt(x2 + z2)
        a1 = x * y * z * np.arcsinh(z / rxy)
        a2 = y / 6 * (3 * z2 - y2) * np.arcsinh(x / ryz)
        a3 = x / 6 * (3 * z2 - x2) * np.arcsinh(y / rxz)
        b1 = z * z2 / 6 * np.arctan(x * y / (z * R))
        b2 = z * y2 / 2 * np.arctan(x * z / (y * R))
        b3 = z * x2 / 2 * np.arctan(y * z / (x * R))
    out = out + np.where(rxy > 0, a1, 0) + np.where(ryz > 0, a2, 0) + np.where(rxz > 0, a3, 0)
    out = out - np.where(z * R > 0, b1, 0) - np.where(y * R > 0, b2, 0) - np.where(x * R > 0, b3, 0)
    return sgn * out


def _second_difference_sum(func, X, Y, Z, dx, dy, dz):
    """sum over e in {-1,0,1}^3 of prod_k w(e_k) * func(X+ex dx, Y+ey dy, Z+ez dz),
    w(0) = 2, w(+-1) = -1 (product of three negated second differences)."""
    acc = 0
    for ex in (-1, 0, 1):
        for ey in (-1, 0, 1):
            for ez in (-1, 0, 1):
                w = (2 if ex == 0 else -1) * (2 if ey == 0 else -1) * (2 if ez == 0 else -1)
                acc = acc + w * func(X + ex * dx, Y + ey * dy, Z + ez * dz)
    return acc


def newell_exact(comp, I, J, K, d, dtype=LD):
    """Exact Newell element ``comp`` at integer cell offsets (I, J, K).

    Evaluated in ``dtype`` (longdouble by default) and returned as float64.
    The offsets I*dx etc. are exact in longdouble for |I| < 2^11 because dx is
    the caller's float64 value."""
    dx, dy, dz = (dtype(v) for v in d)
    X = np.asarray(I).astype(dtype) * dx
    Y = np.asarray(J).astype(dtype) * dy
    Z = np.asarray(K).astype(dtype) * dz
    pi = dtype(np.pi) if dtype is np.float64 else np.arctan(dtype(1)) * 4
    if comp == "xx":
        s = _second_difference_sum(lambda x, y, z: newell_f(x, y, z), X, Y, Z, dx, dy, dz)
    elif comp == "yy":
        s = _second_difference_sum(lambda x, y, z: newell_f(y, z, x), X, Y, Z, dx, dy, dz)
    elif comp == "zz":
        s = _second_difference_sum(lambda x, y, z: newell_f(z, x, y), X, Y, Z, dx, dy, dz)
    elif comp == "xy":
        s = _second_difference_sum(lambda x, y, z: newell_g(x, y, z), X, Y, Z, dx, dy, dz)
    elif comp == "xz":
        s = _second_difference_sum(lambda x, y, z: newell_g(x, z, y), X, Y, Z, dx, dy, dz)
    elif comp == "yz":
        s = _second_difference_sum(lambda x, y, z: newell_g(y, z, x), X, Y, Z, dx, dy, dz)
    else:
        raise ValueError(comp)
    return (s / (4 * pi * dx * dy * dz)).astype(np.float64)


def inverse_r_derivatives(x, y, z, order):
    """All Cartesian derivatives d_x^t d_y^u d_z^v (1/r), t+u+v <= order.

    McMurchie-Davidson recurrence:
        R^(n)_000 = (-1)^n (2n-1)!! / r^(2n+1)
        R^(n)_{t+1,u,v} = t R^(n+1)_{t-1,u,v} + x R^(n+1)_{t,u,v}   (same in u, v)
    and d_x^t d_y^u d_z^v (1/r) = R^(0)_tuv.  Returns a dict (t,u,v) -> array.
    """
    r2 = x * x + y * y + z * z
    r = np.sqrt(r2)

    @lru_cache(maxsize=None)
    def Rn(n, t, u, v):
        if t < 0 or u < 0 or v < 0:
            return 0.0
        if t == 0 and u == 0 and v == 0:
            dfact = 1.0
            for k in range(1, 2 * n, 2):
                dfact *= k
            return (-1) ** n * dfact / (r * r2 ** n)
        if t > 0:
            return (t - 1) * Rn(n + 1, t - 2, u, v) + x * Rn(n + 1, t - 1, u, v)
        if u > 0:
            return (u - 1) * Rn(n + 1, t, u - 2, v) + y * Rn(n + 1, t, u - 1, v)
        return (v - 1) * Rn(n + 1, t, u, v - 2) + z * Rn(n + 1, t, u, v - 1)

    out = {}
    for t in range(order + 1):
        for u in range(order + 1 - t):
            for v in range(order + 1 - t - u):
                out[(t, u, v)] = Rn(0, t, u, v)
    return out


_AXIS = {"x": 0, "y": 1, "z": 2}


def newell_series(comp, I, J, K, d, order=SERIES_ORDER):
    """Far-field Newell element(s) from the tent-moment Taylor series (float64).

    ``comp`` is one component name or a sequence of names (then a list of
    arrays is returned; the derivatives of 1/r are shared)."""
    dx, dy, dz = (float(v) for v in d)
    x = np.asarray(I, dtype=np.float64) * dx
    y = np.asarray(J, dtype=np.float64) * dy
    z = np.asarray(K, dtype=np.float64) * dz
    der = inverse_r_derivatives(x, y, z, 2 * order + 2)

    def C(a, h):
        return 2.0 * h ** (2 * a) / math.factorial(2 * a + 2)

    names = [comp] if isinstance(comp, str) else list(comp)
    res = []
    for name in names:
        base = [0, 0, 0]
        base[_AXIS[name[0]]] += 1
        base[_AXIS[name[1]]] += 1
        acc = np.zeros(np.broadcast(x, y, z).shape)
        for a in range(order + 1):
            for b in range(order + 1 - a):
                for c in range(order + 1 - a - b):
                    key = (base[0] + 2 * a, base[1] + 2 * b, base[2] + 2 * c)
                    acc = acc + C(a, dx) * C(b, dy) * C(c, dz) * der[key]
        res.append(-(dx * dy * dz) / (4 * np.pi) * acc)
    return res[0] if isinstance(comp, str) else res


def is_near(I, J, K, d):
    dmax = max(d)
    r = np.sqrt((np.asarray(I) * d[0]) ** 2 + (np.asarray(J) * d[1]) ** 2 + (np.asarray(K) * d[2]) ** 2)
    return r < NEAR_CELLS * dmax


def newell_tensor(comp, I, J, K, d, chunk=50000):
    """Newell element(s) at integer offsets: exact near, series far (float64).

    ``comp`` is one name or a sequence of names (then a list is returned)."""
    names = [comp] if isinstance(comp, str) else list(comp)
    I, J, K = np.broadcast_arrays(np.asarray(I), np.asarray(J), np.asarray(K))
    shape = I.shape
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    out = [np.empty(I.shape, dtype=np.float64) for _ in names]
    near = is_near(I, J, K, d)
    idx = np.nonzero(near)[0]
    for s in range(0, idx.size, chunk):
        sl = idx[s:s + chunk]
        for o, name in zip(out, names):
            o[sl] = newell_exact(name, I[sl], J[sl], K[sl], d)
    idx = np.nonzero(~near)[0]
    for s in range(0, idx.size, chunk):
        sl = idx[s:s + chunk]
        for o, v in zip(out, newell_series(names, I[sl], J[sl], K[sl], d)):
            o[sl] = v
    out = [o.reshape(shape) for o in out]
    return out[0] if isinstance(comp, str) else out


def offset_grid(n):
    """Integer offsets -(n_k - 1) .. (n_k - 1) per axis, as [z][y][x] index arrays."""
    nx, ny, nz = n
    K, J, I = np.meshgrid(np.arange(-(nz - 1), nz), np.arange(-(ny - 1), ny),
                          np.arange(-(nx - 1), nx), indexing="ij")
    return I, J, K


# parity of each component under i -> -i, j -> -j, k -> -k
PARITY = {"xx": (1, 1, 1), "yy": (1, 1, 1), "zz": (1, 1, 1),
          "xy": (-1, -1, 1), "xz": (-1, 1, -1), "yz": (1, -1, -1)}


def kernel_octant(n, d):
    """The six components at offsets 0 <= i < nx, 0 <= j < ny, 0 <= k < nz,
    as an array [6][nz][ny][nx]."""
    nx, ny, nz = n
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack(newell_tensor(COMPONENTS, I, J, K, d))


def kernel_offsets(n, d):
    """The six Newell components at every offset of an n-cell mesh.

    Returns an array [6][2nz-1][2ny-1][2nx-1], offset (i,j,k) at index
    (k + nz - 1, j + ny - 1, i + nx - 1).  Negative offsets come from the
    non-negative octant by each component's parity (N_xx even in every axis,
    N_xy odd in x and y, ...)."""
    nx, ny, nz = n
    octant = kernel_octant(n, d)
    I, J, K = offset_grid(n)
    out = np.empty((6,) + I.shape)
    for c, name in enumerate(COMPONENTS):
        px, py, pz = PARITY[name]
        sign = (np.where(I < 0, px, 1) * np.where(J < 0, py, 1) * np.where(K < 0, pz, 1))
        out[c] = sign * octant[c][np.abs(K), np.abs(J), np.abs(I)]
    return out
