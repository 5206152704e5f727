"""Micromagnetic fields, LLG and integrators: CPU oracle (test infrastructure only).

Plain float64 numpy restatements of the paper's method, one function per step:

* demag field (Eq. 4): H = -N * M, the linear (non-periodic) convolution of
  M = Ms m with the Newell tensor; once as an O(N^2) direct sum and once with
  numpy's FFT on the grid zero-padded to 2n per axis (1 when n = 1);
* exchange field (Eq. 2) with the magnetisation read as the unit vector m:
  H_i = 2 / (mu0 Ms_i) * sum_nb A_i,nb (m_nb - m_i) / d_axis^2, A_i,nb the
  harmonic mean, free (Neumann) boundary, Ms = 0 cells are vacuum;
* uniaxial anisotropy H = 2 Ku / (mu0 Ms) (m.u) u and a uniform Zeeman field
  (both named in the paper's Implementation section, formulas standard);
* the LLG right-hand side (Eq. 1) for unit m:
  dm/dt = -gamma / (1 + alpha^2) [m x H + alpha m x (m x H)];
* classic RK4 and Fehlberg's RKF45 (the paper's integrator, Implementation
  section), error = max over cells of |m5 - m4|, 4th-order solution propagated,
  m renormalised after every accepted step;
* energies, maximum torque and relax().

Layout: vectors are arrays [3][nz][ny][nx] (x fastest); scalars [nz][ny][nx].
"""

import numpy as np

from . import newell

MU0 = 4e-7 * np.pi
GAMMA = 2.2127615e5          # mu0 * gamma_e, m / (A s)
HBAR = 1.054571817e-34       # J s (exact SI value of h / 2 pi)
QE = 1.602176634e-19         # C (exact SI value)


class Problem:
    """Mesh + material: the state an ``mm_ctx`` holds on the GPU side."""

    def __init__(self, n, d, Ms=8e5, A=1.3e-11, alpha=0.02, Ku=0.0, u=(0.0, 0.0, 1.0),
                 h_ext=(0.0, 0.0, 0.0), Ms_cell=None, A_cell=None, D=0.0, dmi="interfacial", stt=None):
        self.n = tuple(int(v) for v in n)
        self.d = tuple(float(v) for v in d)
        nx, ny, nz = self.n
        shape = (nz, ny, nx)
        self.Ms = np.broadcast_to(np.asarray(Ms if Ms_cell is None else Ms_cell, dtype=np.float64), shape).copy()
        self.A = np.broadcast_to(np.asarray(A if A_cell is None else A_cell, dtype=np.float64), shape).copy()
        self.alpha = float(alpha)
        self.Ku = float(Ku)
        u = np.asarray(u, dtype=np.float64)
        self.u = u / np.linalg.norm(u)
        self.h_ext = np.asarray(h_ext, dtype=np.float64)
        self.D = float(D)
        assert dmi in ("interfacial", "bulk")
        self.dmi_type = dmi
        # Slonczewski spin-transfer torque: dict(J, P, Lambda, eps_prime, p, d) or None
        self.stt = None
        if stt is not None:
            st = dict(stt)
            pv = np.asarray(st["p"], dtype=np.float64)
            st["p"] = pv / np.linalg.norm(pv)
            st.setdefault("d", self.n[2] * self.d[2])
            self.stt = st
        self._kernel = None
        # the FFT namespace (rfftn / irfftn) the convolution uses: numpy's by
        # default; a timing harness may substitute a multi-threaded one with
        # the same functions (same transforms, different thread count)
        self.fft = np.fft

    @property
    def V(self):
        return self.d[0] * self.d[1] * self.d[2]

    @property
    def padded(self):
        return tuple(2 * v if v > 1 else 1 for v in self.n)

    # ------------------------------------------------------------- demag
    def kernel(self):
        """Real-space Newell tensor at all offsets, [6][2nz-1][2ny-1][2nx-1]."""
        if self._kernel is None:
            self._kernel = newell.kernel_offsets(self.n, self.d)
        return self._kernel

    def kernel_hat(self):
        """FFT of the kernel placed on the padded grid (offset o at index o mod P)."""
        nx, ny, nz = self.n
        Px, Py, Pz = self.padded
        Kr = self.kernel()
        out = []
        for c in range(6):
            grid = np.zeros((Pz, Py, Px))
            grid[np.ix_(np.arange(-(nz - 1), nz) % Pz, np.arange(-(ny - 1), ny) % Py,
                        np.arange(-(nx - 1), nx) % Px)] = Kr[c]
            out.append(self.fft.rfftn(grid, axes=(0, 1, 2)))
        return out

    def demag_fft(self, m):
        """H = -N * (Ms m), zero-padded FFT convolution in float64."""
        nx, ny, nz = self.n
        Px, Py, Pz = self.padded
        Nh = self.kernel_hat()
        Mh = [self.fft.rfftn(self.Ms * m[c], s=(Pz, Py, Px), axes=(0, 1, 2)) for c in range(3)]
        xx, yy, zz, xy, xz, yz = Nh
        T = [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]
        H = np.empty_like(m, dtype=np.float64)
        for i in range(3):
            Hh = -(T[i][0] * Mh[0] + T[i][1] * Mh[1] + T[i][2] * Mh[2])
            H[i] = self.fft.irfftn(Hh, s=(Pz, Py, Px), axes=(0, 1, 2))[:nz, :ny, :nx]
        return H

    def demag_direct(self, m, targets=None):
        """O(N^2) direct sum H_i = -sum_j N(r_i - r_j) Ms_j m_j.

        ``targets``: optional list of (x, y, z) cells; returns [3][len] then."""
        nx, ny, nz = self.n
        Kr = self.kernel()
        M = self.Ms * m
        if targets is None:
            targets = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
            full = True
        else:
            full = False
        out = np.zeros((3, len(targets)))
        T = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
        for t, (x, y, z) in enumerate(targets):
            # offset (x - xs) at index (x - xs) + n - 1; sources xs = 0..n-1
            sx = slice(x + nx - 1, x - 1 if x > 0 else None, -1)
            sy = slice(y + ny - 1, y - 1 if y > 0 else None, -1)
            sz = slice(z + nz - 1, z - 1 if z > 0 else None, -1)
            for i in range(3):
                acc = 0.0
                for j in range(3):
                    acc += np.sum(Kr[T[i][j]][sz, sy, sx] * M[j])
                out[i, t] = -acc
        if full:
            return out.reshape(3, nz, ny, nx)
        return out

    # ---------------------------------------------------------- exchange
    def exchange(self, m):
        """6-point exchange field, harmonic-mean A, Neumann boundary, vacuum Ms = 0."""
        H = np.zeros_like(m, dtype=np.float64)
        Ms, A = self.Ms, self.A
        mag = Ms > 0
        for axis, h in ((2, self.d[0]), (1, self.d[1]), (0, self.d[2])):
            for shift in (1, -1):
                n_ax = Ms.shape[axis]
                if n_ax == 1:
                    continue
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if shift == 1:      # neighbour at +1 along axis
                    dst[axis] = slice(0, n_ax - 1)
                    src[axis] = slice(1, n_ax)
                else:
                    dst[axis] = slice(1, n_ax)
                    src[axis] = slice(0, n_ax - 1)
                dst, src = tuple(dst), tuple(src)
                Ai, An = A[dst], A[src]
                with np.errstate(divide="ignore", invalid="ignore"):
                    Ah = np.where(Ai + An > 0, 2 * Ai * An / (Ai + An), 0.0)
                w = Ah * mag[src] * mag[dst] / (h * h)
                for c in range(3):
                    H[c][dst] += w * (m[c][src] - m[c][dst])
        with np.errstate(divide="ignore", invalid="ignore"):
            pref = np.where(mag, 2.0 / (MU0 * Ms), 0.0)
        return H * pref

    def dmi_vectors(self):
        """e_k^DMI for k = x, y, z (Eq. 3): (e_y, -e_x, 0) interfacial, (e_x, e_y, e_z) bulk."""
        ex, ey, ez = np.eye(3)
        if self.dmi_type == "interfacial":
            return [ey, -ex, np.zeros(3)]
        return [ex, ey, ez]

    def dmi(self, m):
        """Eq. 3 for unit m: H = 2D / (mu0 Ms) sum_k e_k x dm/dk, dm/dk by the
        central difference (m[+k] - m[-k]) / (2 d_k) with a neighbour outside
        the magnet (mesh edge or Ms = 0) contributing nothing: the field of the
        bond energy (D V / d_k) sum_bonds e_k . (m_i x m_(i+k))."""
        H = np.zeros_like(m, dtype=np.float64)
        if self.D == 0.0:
            return H
        Ms = self.Ms
        mag = Ms > 0
        evec = self.dmi_vectors()
        for k, (axis, h) in enumerate(((2, self.d[0]), (1, self.d[1]), (0, self.d[2]))):
            e = evec[k]
            n_ax = Ms.shape[axis]
            if n_ax == 1 or not e.any():
                continue
            for shift in (1, -1):
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if shift == 1:
                    dst[axis], src[axis] = slice(0, n_ax - 1), slice(1, n_ax)
                else:
                    dst[axis], src[axis] = slice(1, n_ax), slice(0, n_ax - 1)
                dst, src = tuple(dst), tuple(src)
                w = shift * mag[src] * mag[dst] / (2 * h)
                nb = np.stack([m[c][src] for c in range(3)])
                cr = np.cross(np.broadcast_to(e[:, None, None, None], nb.shape), nb, axis=0)
                for c in range(3):
                    H[c][dst] += w * cr[c]
        with np.errstate(divide="ignore", invalid="ignore"):
            pref = np.where(mag, 2.0 * self.D / (MU0 * Ms), 0.0)
        return H * pref

    def dmi_bond_energy(self, m):
        """(D V / d_k) sum over bonds (i, i + k) between magnetic cells of
        e_k . (m_i x m_(i+k)): the energy whose field is Eq. 3 discretised."""
        if self.D == 0.0:
            return 0.0
        mag = self.Ms > 0
        E = 0.0
        for k, (axis, h) in enumerate(((2, self.d[0]), (1, self.d[1]), (0, self.d[2]))):
            e = self.dmi_vectors()[k]
            n_ax = mag.shape[axis]
            if n_ax == 1:
                continue
            a = [slice(None)] * 3
            b = [slice(None)] * 3
            a[axis], b[axis] = slice(0, n_ax - 1), slice(1, n_ax)
            a, b = tuple(a), tuple(b)
            mi = np.stack([m[c][a] for c in range(3)])
            mj = np.stack([m[c][b] for c in range(3)])
            cr = np.cross(mi, mj, axis=0)
            E += np.sum((e[0] * cr[0] + e[1] * cr[1] + e[2] * cr[2]) * mag[a] * mag[b]) * self.D * self.V / h
        return float(E)

    def anisotropy(self, m):
        mag = self.Ms > 0
        with np.errstate(divide="ignore", invalid="ignore"):
            pref = np.where(mag, 2 * self.Ku / (MU0 * self.Ms), 0.0)
        mu = self.u[0] * m[0] + self.u[1] * m[1] + self.u[2] * m[2]
        return np.stack([pref * mu * self.u[c] for c in range(3)])

    def zeeman(self, m):
        mag = (self.Ms > 0).astype(np.float64)
        return np.stack([mag * self.h_ext[c] for c in range(3)])

    def h_eff(self, m, demag=None):
        Hd = self.demag_fft(m) if demag is None else demag
        return Hd + self.exchange(m) + self.anisotropy(m) + self.zeeman(m) + self.dmi(m)

    # --------------------------------------------------------------- LLG
    def llg_rhs(self, m, H):
        """Eq. 1 for the unit vector m (cells with Ms = 0 do not move), plus
        the Slonczewski torque when configured."""
        mxh = np.cross(m, H, axis=0)
        mxmxh = np.cross(m, mxh, axis=0)
        pref = -GAMMA / (1 + self.alpha ** 2)
        r = pref * (mxh + self.alpha * mxmxh)
        if self.stt is not None:
            r = r + self.stt_torque(m)
        return r * (self.Ms > 0)

    def stt_torque(self, m):
        """Slonczewski spin-transfer torque (named in the paper as a local
        term; reading taken): in Gilbert form the term
        gamma beta [eps m x (p x m) + eps' p x m] is added to Eq. 1 with
        beta = hbar J / (mu0 e Ms d) (A/m), eps = P L^2 / ((L^2 + 1) + (L^2 - 1) m.p);
        solved for dm/dt it becomes
        gamma beta / (1 + alpha^2) [(eps + alpha eps') m x (p x m) - (eps' - alpha eps) m x p]."""
        st = self.stt
        pv = st["p"].reshape(3, 1, 1, 1) * np.ones_like(m)
        mag = self.Ms > 0
        with np.errstate(divide="ignore", invalid="ignore"):
            beta = np.where(mag, HBAR * st["J"] / (MU0 * QE * np.where(mag, self.Ms, 1.0) * st["d"]), 0.0)
        L2 = st["Lambda"] ** 2
        mp = np.sum(m * pv, axis=0)
        eps = st["P"] * L2 / ((L2 + 1) + (L2 - 1) * mp)
        a = self.alpha
        pxm = np.cross(pv, m, axis=0)
        mxpxm = np.cross(m, pxm, axis=0)
        mxp = -pxm
        c = GAMMA * beta / (1 + a * a)
        return c * ((eps + a * st["eps_prime"]) * mxpxm - (st["eps_prime"] - a * eps) * mxp)

    def rhs(self, m):
        return self.llg_rhs(m, self.h_eff(m))

    def normalise(self, m):
        nrm = np.sqrt(np.sum(m * m, axis=0))
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where((self.Ms > 0) & (nrm > 0), m / nrm, 0.0 * m)

    def rk4_step(self, m, dt):
        """Classic 4-stage Runge-Kutta step, then renormalise."""
        k1 = self.rhs(m)
        k2 = self.rhs(m + dt / 2 * k1)
        k3 = self.rhs(m + dt / 2 * k2)
        k4 = self.rhs(m + dt * k3)
        return self.normalise(m + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4))

    def rkf45_trial(self, m, dt):
        """One Fehlberg 4(5) trial step.  Returns (m4 renormalised, err).

        err = max over cells of |m5 - m4| = dt * max |sum_j (b5_j - b4_j) k_j|."""
        A, B4, B5 = FEHLBERG_A, FEHLBERG_B4, FEHLBERG_B5
        k = []
        for s in range(6):
            ms = m.copy()
            for j in range(s):
                ms = ms + dt * A[s][j] * k[j]
            k.append(self.rhs(ms))
        m4 = m.copy()
        e = np.zeros_like(m)
        for j in range(6):
            m4 = m4 + dt * B4[j] * k[j]
            e = e + (B5[j] - B4[j]) * k[j]
        err = dt * float(np.max(np.sqrt(np.sum(e * e, axis=0)))) if e.size else 0.0
        return self.normalise(m4), err

    # ---------------------------------------------------------- energies
    def energies(self, m):
        """(E_demag, E_exchange, E_anisotropy, E_zeeman, E_dmi) in J."""
        V = self.V
        Ms = self.Ms
        e_d = -0.5 * MU0 * V * np.sum(Ms * np.sum(m * self.demag_fft(m), axis=0))
        e_x = -0.5 * MU0 * V * np.sum(Ms * np.sum(m * self.exchange(m), axis=0))
        mu = self.u[0] * m[0] + self.u[1] * m[1] + self.u[2] * m[2]
        e_a = -self.Ku * V * np.sum((Ms > 0) * mu * mu)
        e_z = -MU0 * V * np.sum(Ms * np.sum(m * self.zeeman(m), axis=0))
        e_m = -0.5 * MU0 * V * np.sum(Ms * np.sum(m * self.dmi(m), axis=0))
        return np.array([e_d, e_x, e_a, e_z, e_m])

    def max_torque(self, m, H=None):
        """max over magnetic cells of |m x H_eff| / Ms (dimensionless)."""
        H = self.h_eff(m) if H is None else H
        t = np.sqrt(np.sum(np.cross(m, H, axis=0) ** 2, axis=0))
        mag = self.Ms > 0
        return float(np.max(np.where(mag, t / np.where(mag, self.Ms, 1.0), 0.0)))


# Fehlberg's RKF45 tableau (Fehlberg 1969): stage matrix, 4th- and 5th-order weights.
FEHLBERG_A = [
    [],
    [1 / 4],
    [3 / 32, 9 / 32],
    [1932 / 2197, -7200 / 2197, 7296 / 2197],
    [439 / 216, -8.0, 3680 / 513, -845 / 4104],
    [-8 / 27, 2.0, -3544 / 2565, 1859 / 4104, -11 / 40],
]
FEHLBERG_C = [0.0, 1 / 4, 3 / 8, 12 / 13, 1.0, 1 / 2]
FEHLBERG_B4 = [25 / 216, 0.0, 1408 / 2565, 2197 / 4104, -1 / 5, 0.0]
FEHLBERG_B5 = [16 / 135, 0.0, 6656 / 12825, 28561 / 56430, -9 / 50, 2 / 55]

# step-size control (reading of the paper's RKF45, which names the method only)
SAFETY, SHRINK_MIN, GROW_MAX, DT_FLOOR = 0.9, 0.2, 5.0, 1e-20


def next_dt(dt, err, tol):
    """dt * clamp(0.9 (tol / err)^(1/5), 0.2, 5)."""
    if err <= 0.0:
        return dt * GROW_MAX
    return dt * min(GROW_MAX, max(SHRINK_MIN, SAFETY * (tol / err) ** 0.2))


def rkf45_step(p, m, t, dt, tol):
    """Adaptive step: retry with smaller dt until accepted.

    Returns (m_new, t_new, dt_next, err, n_rejected)."""
    rejected = 0
    while True:
        m4, err = p.rkf45_trial(m, dt)
        if err <= tol:
            return m4, t + dt, next_dt(dt, err, tol), err, rejected
        rejected += 1
        dt = next_dt(dt, err, tol)
        if dt < DT_FLOOR:
            raise FloatingPointError("dt underflow")


def relax(p, m, t_max, torque_tol, max_steps, dt0=1e-14, tol=1e-5):
    """RKF45 LLG until max |m x H| / Ms <= torque_tol, t >= t_max or max_steps."""
    t, dt, steps = 0.0, dt0, 0
    while steps < max_steps and t < t_max:
        if p.max_torque(m) <= torque_tol:
            break
        dt = min(dt, t_max - t)
        m, t, dt, _, _ = rkf45_step(p, m, t, dt, tol)
        steps += 1
    return m, t, steps


# Barzilai-Borwein energy minimisation.  The paper names the method (its
# RKF45 paragraph, and the minimiser call of its example script) without
# printing it; the reading taken here is steepest descent on the unit
# sphere with Barzilai-Borwein step lengths, alternating the two quotients,
# and a full step (tau_max) where the path meets non-positive curvature
# (resetting to the small first step there stalls on saddles).
BB_TAU0, BB_TAU_MAX = 1e-4, 1.0


def minimize_bb(p, m, torque_tol, max_iter, tau0=BB_TAU0, tau_max=BB_TAU_MAX):
    """Minimise the energy over unit m.  Per iteration k: h = H_eff / Ms
    (zero on vacuum cells), g = m x (m x h) (the descent direction is -g,
    the component of h perpendicular to m), m <- normalise(m - tau g).
    tau = tau0 on the first step; afterwards, with s = m_k - m_(k-1),
    y = g_k - g_(k-1) summed over all cells and components,
    tau = (s.s)/(s.y) on odd k and (s.y)/(y.y) on even k, or tau_max when
    the quotient is not a positive finite number.  Stops before a step once
    max |m x H_eff| / Ms <= torque_tol, or after max_iter steps.
    Returns (m, steps taken)."""
    mag = p.Ms > 0
    inv_ms = np.where(mag, 1.0 / np.where(mag, p.Ms, 1.0), 0.0)
    m_prev = g_prev = None
    tau = tau0
    for k in range(max_iter + 1):
        H = p.h_eff(m)
        if p.max_torque(m, H) <= torque_tol or k == max_iter:
            return m, k
        h = H * inv_ms
        g = np.cross(m, np.cross(m, h, axis=0), axis=0)
        if m_prev is not None:
            s_, y_ = m - m_prev, g - g_prev
            ss, sy, yy = float(np.sum(s_ * s_)), float(np.sum(s_ * y_)), float(np.sum(y_ * y_))
            with np.errstate(divide="ignore", invalid="ignore"):
                tau = ss / sy if k % 2 == 1 else sy / yy
            if not (np.isfinite(tau) and tau > 0):
                tau = tau_max
        m_prev, g_prev = m, g
        m = p.normalise(m - tau * g)
    return m, max_iter
