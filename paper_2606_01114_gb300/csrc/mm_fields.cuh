// Per-cell field helpers shared by the LLG kernels and their adjoints:
// material parameters, the 6-point exchange stencil (Eq. 2 for unit m),
// anisotropy + Zeeman, and the LLG right-hand side (Eq. 1 for unit m).
#pragma once

#include "mm_internal.cuh"

namespace mm {

// --------------------------------------------------------- parameters
template <typename T> struct Params {
    int nx, ny, nz;
    long N;
    const T* Ms_cell;   // nullable
    const T* A_cell;    // nullable
    T Ms, A;
    T cx, cy, cz;       // 2 / (mu0 d^2) per axis
    T anis;             // 2 Ku / mu0
    T ux, uy, uz;
    T hx, hy, hz;
    T pref;             // -gamma / (1 + alpha^2)
    T alpha;
    int dmi;            // 0 none, 1 interfacial, 2 bulk
    T dx_c, dy_c, dz_c; // D / (mu0 d) per axis
    int stt;            // Slonczewski torque on
    T stt_c;            // gamma hbar J / (mu0 e d (1 + alpha^2)); divided by Ms per cell
    T stt_P, stt_L2, stt_eps2;
    T px, py, pz;
};

template <typename T>
inline Params<T> make_params(const mm_ctx* ctx) {
    Params<T> p;
    p.nx = ctx->nx;
    p.ny = ctx->ny;
    p.nz = ctx->nz;
    p.N = ctx->N;
    p.Ms_cell = ctx->has_Ms_cell ? (const T*)ctx->Ms_cell : nullptr;
    p.A_cell = ctx->has_A_cell ? (const T*)ctx->A_cell : nullptr;
    p.Ms = (T)ctx->Ms;
    p.A = (T)ctx->A;
    p.cx = (T)(2.0 / (kMu0 * ctx->dx * ctx->dx));
    p.cy = (T)(2.0 / (kMu0 * ctx->dy * ctx->dy));
    p.cz = (T)(2.0 / (kMu0 * ctx->dz * ctx->dz));
    p.anis = (T)(2.0 * ctx->Ku / kMu0);
    p.ux = (T)ctx->u[0];
    p.uy = (T)ctx->u[1];
    p.uz = (T)ctx->u[2];
    p.hx = (T)ctx->hext[0];
    p.hy = (T)ctx->hext[1];
    p.hz = (T)ctx->hext[2];
    p.pref = (T)(-kGamma / (1.0 + ctx->alpha * ctx->alpha));
    p.alpha = (T)ctx->alpha;
    p.dmi = ctx->D != 0.0 ? ctx->dmi_type : 0;
    p.dx_c = (T)(ctx->D / (kMu0 * ctx->dx));
    p.dy_c = (T)(ctx->D / (kMu0 * ctx->dy));
    p.dz_c = (T)(ctx->D / (kMu0 * ctx->dz));
    p.stt = ctx->stt_on;
    p.stt_c = (T)(kGamma * kHbar * ctx->stt_J / (kMu0 * kQe * ctx->stt_d * (1.0 + ctx->alpha * ctx->alpha)));
    p.stt_P = (T)ctx->stt_P;
    p.stt_L2 = (T)(ctx->stt_L * ctx->stt_L);
    p.stt_eps2 = (T)ctx->stt_eps2;
    p.px = (T)ctx->stt_p[0];
    p.py = (T)ctx->stt_p[1];
    p.pz = (T)ctx->stt_p[2];
    return p;
}

template <typename T> struct V3 { T x, y, z; };

template <typename T>
__device__ __forceinline__ V3<T> load3(const T* __restrict__ a, long i, long N) {
    return {a[i], a[i + N], a[i + 2 * N]};
}
template <typename T>
__device__ __forceinline__ void store3(T* __restrict__ a, long i, long N, V3<T> v) {
    a[i] = v.x;
    a[i + N] = v.y;
    a[i + 2 * N] = v.z;
}

// exchange field at cell i (x, y, z) of state m; Msi > 0
template <typename T>
__device__ __forceinline__ V3<T> exchange_at(const Params<T>& p, const T* __restrict__ m, long i, int x, int y,
                                             int z, V3<T> mi, T Msi) {
    const T Ai = p.A_cell ? p.A_cell[i] : p.A;
    T ax = 0, ay = 0, az = 0;
    auto nb = [&](long j, T c) {
        T Msj = p.Ms_cell ? p.Ms_cell[j] : p.Ms;
        if (Msj == (T)0) return;
        T Ah;
        if (p.A_cell) {
            T Aj = p.A_cell[j];
            T s = Ai + Aj;
            Ah = s > (T)0 ? (T)2 * Ai * Aj / s : (T)0;
        } else {
            Ah = p.A;
        }
        T w = Ah * c;
        ax += w * (m[j] - mi.x);
        ay += w * (m[j + p.N] - mi.y);
        az += w * (m[j + 2 * p.N] - mi.z);
    };
    const long sx = 1, sy = p.nx, sz = (long)p.nx * p.ny;
    if (x > 0) nb(i - sx, p.cx);
    if (x < p.nx - 1) nb(i + sx, p.cx);
    if (y > 0) nb(i - sy, p.cy);
    if (y < p.ny - 1) nb(i + sy, p.cy);
    if (z > 0) nb(i - sz, p.cz);
    if (z < p.nz - 1) nb(i + sz, p.cz);
    T inv = (T)1 / Msi;
    return {ax * inv, ay * inv, az * inv};
}

// anisotropy + Zeeman at a magnetic cell
template <typename T>
__device__ __forceinline__ V3<T> local_at(const Params<T>& p, V3<T> mi, T Msi) {
    T mu = mi.x * p.ux + mi.y * p.uy + mi.z * p.uz;
    T k = p.anis / Msi * mu;
    return {k * p.ux + p.hx, k * p.uy + p.hy, k * p.uz + p.hz};
}

// DMI field (Eq. 3) at cell i of unit m; Msi > 0:
//   H = 2 D / (mu0 Ms) sum_k e_k x (m[+k] - m[-k]) / (2 d_k),
// e_k = (e_y, -e_x, 0) interfacial or (e_x, e_y, e_z) bulk; a neighbour
// outside the magnet (mesh edge or Ms = 0) contributes nothing (the field
// of the bond energy (D V / d_k) sum_bonds e_k . (m_i x m_(i+k))).
template <typename T>
__device__ __forceinline__ V3<T> dmi_at(const Params<T>& p, const T* __restrict__ m, long i, int x, int y, int z,
                                        T Msi) {
    T hx = 0, hy = 0, hz = 0;
    // sum over the present neighbours of sign * (m_nb) per axis: v_axis
    auto acc = [&](long j, T sgn, T& vx, T& vy, T& vz) {
        if (p.Ms_cell && p.Ms_cell[j] == (T)0) return;
        vx += sgn * m[j];
        vy += sgn * m[j + p.N];
        vz += sgn * m[j + 2 * p.N];
    };
    const long sx = 1, sy = p.nx, sz = (long)p.nx * p.ny;
    T ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0, cx = 0, cy = 0, cz = 0;
    if (x < p.nx - 1) acc(i + sx, (T)1, ax, ay, az);
    if (x > 0) acc(i - sx, (T)-1, ax, ay, az);
    if (y < p.ny - 1) acc(i + sy, (T)1, bx, by, bz);
    if (y > 0) acc(i - sy, (T)-1, bx, by, bz);
    if (p.dmi == 2) {
        if (z < p.nz - 1) acc(i + sz, (T)1, cx, cy, cz);
        if (z > 0) acc(i - sz, (T)-1, cx, cy, cz);
    }
    if (p.dmi == 1) {
        // e_y x a (x axis) and -e_x x b (y axis)
        hx = p.dx_c * az;
        hz = -p.dx_c * ax;
        hy = p.dy_c * bz;
        hz += -p.dy_c * by;
    } else {
        // e_x x a, e_y x b, e_z x c
        hy = -p.dx_c * az;
        hz = p.dx_c * ay;
        hx = p.dy_c * bz;
        hz += -p.dy_c * bx;
        hx += -p.dz_c * cy;
        hy += p.dz_c * cx;
    }
    const T inv = (T)1 / Msi;
    return {hx * inv, hy * inv, hz * inv};
}

// Slonczewski spin-transfer torque (a local term beside Eq. 1; the form is
// the reading taken): the Gilbert-form term gamma beta [eps m x (p x m) +
// eps' p x m], beta = hbar J / (mu0 e Ms d), eps = P L^2 / ((L^2 + 1) +
// (L^2 - 1) m.p), solved for dm/dt:
//   gamma beta / (1 + alpha^2) [(eps + alpha eps') m x (p x m) - (eps' - alpha eps) m x p]
template <typename T>
__device__ __forceinline__ V3<T> stt_at(const Params<T>& p, V3<T> m, T Msi) {
    const T mp = m.x * p.px + m.y * p.py + m.z * p.pz;
    const T eps = p.stt_P * p.stt_L2 / ((p.stt_L2 + (T)1) + (p.stt_L2 - (T)1) * mp);
    const T c = p.stt_c / Msi;
    const T a = c * (eps + p.alpha * p.stt_eps2), b = c * (p.stt_eps2 - p.alpha * eps);
    // m x (p x m) = (m.m) p - (m.p) m (stage states are not unit vectors);  m x p
    const T mm = m.x * m.x + m.y * m.y + m.z * m.z;
    const V3<T> dl = {mm * p.px - mp * m.x, mm * p.py - mp * m.y, mm * p.pz - mp * m.z};
    const V3<T> mxp = {m.y * p.pz - m.z * p.py, m.z * p.px - m.x * p.pz, m.x * p.py - m.y * p.px};
    return {a * dl.x - b * mxp.x, a * dl.y - b * mxp.y, a * dl.z - b * mxp.z};
}

template <typename T>
__device__ __forceinline__ V3<T> llg_rhs(const Params<T>& p, V3<T> m, V3<T> H) {
    V3<T> a = {m.y * H.z - m.z * H.y, m.z * H.x - m.x * H.z, m.x * H.y - m.y * H.x};   // m x H
    V3<T> b = {m.y * a.z - m.z * a.y, m.z * a.x - m.x * a.z, m.x * a.y - m.y * a.x};   // m x (m x H)
    return {p.pref * (a.x + p.alpha * b.x), p.pref * (a.y + p.alpha * b.y), p.pref * (a.z + p.alpha * b.z)};
}

__device__ __forceinline__ void decompose(long i, int nx, int ny, int& x, int& y, int& z) {
    x = (int)(i % nx);
    long r = i / nx;
    y = (int)(r % ny);
    z = (int)(r / ny);
}

}  // namespace mm
