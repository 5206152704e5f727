// K1: the Newell demagnetisation tensor on the device.
//
// The paper convolves M with a kernel N computed by Newell's formula
// (Implementation section, Eq. 4).  N_ij at a cell offset is the 27-point
// product of second differences (weights -1, 2, -1 per axis) of Newell's
// auxiliary functions f (diagonal components) and g (off-diagonal ones),
// divided by 4 pi dx dy dz, with H = -N M (self term 1/3 for a cube).
//
// The 27-point sum cancels about R^6 units of roundoff at a distance of R
// cells, so plain FP64 loses up to ~1e-10 of the field.  Everything here runs
// in double-double arithmetic (about 106 significant bits) built from FP64
// error-free transformations:
//   two-sum (Knuth), fast two-sum (Dekker), two-product via fma;
//   division by two Newton corrections, square root by one Newton step;
//   log(a) = e ln 2 + 2 atanh(s), s = (m-1)/(m+1), m in [1/sqrt2, sqrt2),
//     atanh summed as its Taylor series (|s| <= 0.172, 24 terms);
//   atan(t) reduced to t <= 1 by atan(t) = pi/2 - atan(1/t), then three
//     half-angle steps t -> t / (1 + sqrt(1 + t^2)), then its Taylor series
//     (t <= 0.099, 19 terms) times 8;
//   asinh(t) = log(t + sqrt(t^2 + 1)) for t >= 0.
// Coordinates i*dx are formed exactly (two-product), so the only error left
// in N is the final rounding to FP64 (plus ~1e-30 relative series error).
// f and g are evaluated once per grid point (|i| <= nx, ...) and the
// second differences gathered from that grid with each function's parity.
//
// This translation unit is compiled with -fmad=false so that no multiply-add
// contraction breaks the error-free transformations.
#include "mm_internal.cuh"

namespace mm {
namespace {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ dd ddc(double a) { return {a, 0.0}; }
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo;
    p.lo += a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, ddc(q3));
}
__device__ __forceinline__ dd dd_sqrt(dd a) {
    if (a.hi <= 0.0) return ddc(0.0);
    double x = sqrt(a.hi);
    dd x2 = two_prod(x, x);
    double corr = (((a.hi - x2.hi) - x2.lo) + a.lo) / (2.0 * x);
    return fast_two_sum(x, corr);
}

__device__ const dd kLn2 = {0.6931471805599453, 2.3190468138462996e-17};
__device__ const dd kPiDD = {3.141592653589793, 1.2246467991473532e-16};
__device__ const dd kPi2 = {1.5707963267948966, 6.123233995736766e-17};

constexpr int kLogTerms = 24;
constexpr int kAtanTerms = 19;
// 1 / (2n + 1) in double-double, filled once by init_inv_odd
__device__ dd g_inv_odd[32];

__global__ void init_inv_odd() {
    int n = threadIdx.x;
    if (n < 32) g_inv_odd[n] = dd_div(ddc(1.0), ddc(2.0 * n + 1.0));
}

__device__ dd dd_log(dd a) {   // a > 0
    int e;
    double m = frexp(a.hi, &e);   // a.hi = m 2^e, m in [0.5, 1)
    if (m < 0.70710678118654752) e -= 1;
    dd am = {ldexp(a.hi, -e), ldexp(a.lo, -e)};
    dd s = dd_div(dd_sub(am, ddc(1.0)), dd_add(am, ddc(1.0)));
    dd s2 = dd_mul(s, s);
    dd acc = g_inv_odd[kLogTerms];
    for (int n = kLogTerms - 1; n >= 0; --n) acc = dd_add(dd_mul(acc, s2), g_inv_odd[n]);
    dd lm = dd_mul_d(dd_mul(s, acc), 2.0);
    return dd_add(dd_mul_d(kLn2, (double)e), lm);
}

__device__ dd dd_asinh(dd t) {   // t >= 0
    if (t.hi == 0.0) return ddc(0.0);
    dd r = dd_sqrt(dd_add(dd_mul(t, t), ddc(1.0)));
    return dd_log(dd_add(t, r));
}

__device__ dd dd_atan(dd t) {    // t >= 0
    if (t.hi == 0.0) return ddc(0.0);
    bool inv = t.hi > 1.0;
    if (inv) t = dd_div(ddc(1.0), t);
    for (int h = 0; h < 3; ++h)
        t = dd_div(t, dd_add(ddc(1.0), dd_sqrt(dd_add(ddc(1.0), dd_mul(t, t)))));
    dd t2 = dd_mul(t, t);
    dd acc = (kAtanTerms & 1) ? dd_neg(g_inv_odd[kAtanTerms]) : g_inv_odd[kAtanTerms];
    for (int n = kAtanTerms - 1; n >= 0; --n) {
        dd c = (n & 1) ? dd_neg(g_inv_odd[n]) : g_inv_odd[n];
        acc = dd_add(dd_mul(acc, t2), c);
    }
    dd r = dd_mul_d(dd_mul(t, acc), 8.0);
    return inv ? dd_sub(kPi2, r) : r;
}

// Newell's f(x, y, z) for x, y, z >= 0 (even in every argument).
__device__ dd newell_f(dd x, dd y, dd z) {
    dd x2 = dd_mul(x, x), y2 = dd_mul(y, y), z2 = dd_mul(z, z);
    dd R = dd_sqrt(dd_add(dd_add(x2, y2), z2));
    // (2x^2 - y^2 - z^2) R / 6
    dd out = dd_div(dd_mul(dd_sub(dd_sub(dd_mul_d(x2, 2.0), y2), z2), R), ddc(6.0));
    dd xz2 = dd_add(x2, z2), xy2 = dd_add(x2, y2);
    if (xz2.hi > 0.0 && y.hi > 0.0) {
        dd a = dd_asinh(dd_div(y, dd_sqrt(xz2)));
        out = dd_add(out, dd_mul(dd_mul_d(dd_mul(y, dd_sub(z2, x2)), 0.5), a));
    }
    if (xy2.hi > 0.0 && z.hi > 0.0) {
        dd a = dd_asinh(dd_div(z, dd_sqrt(xy2)));
        out = dd_add(out, dd_mul(dd_mul_d(dd_mul(z, dd_sub(y2, x2)), 0.5), a));
    }
    if (x.hi > 0.0 && y.hi > 0.0 && z.hi > 0.0) {
        dd a = dd_atan(dd_div(dd_mul(y, z), dd_mul(x, R)));
        out = dd_sub(out, dd_mul(dd_mul(dd_mul(x, y), z), a));
    }
    return out;
}

// Newell's g(x, y, z) for x, y, z >= 0 (odd in x and y, even in z).
__device__ dd newell_g(dd x, dd y, dd z) {
    dd x2 = dd_mul(x, x), y2 = dd_mul(y, y), z2 = dd_mul(z, z);
    dd R = dd_sqrt(dd_add(dd_add(x2, y2), z2));
    dd out = dd_neg(dd_div(dd_mul(dd_mul(x, y), R), ddc(3.0)));
    dd xy2 = dd_add(x2, y2), yz2 = dd_add(y2, z2), xz2 = dd_add(x2, z2);
    if (xy2.hi > 0.0 && x.hi > 0.0 && y.hi > 0.0 && z.hi > 0.0) {
        dd a = dd_asinh(dd_div(z, dd_sqrt(xy2)));
        out = dd_add(out, dd_mul(dd_mul(dd_mul(x, y), z), a));
    }
    if (yz2.hi > 0.0 && y.hi > 0.0 && x.hi > 0.0) {
        dd a = dd_asinh(dd_div(x, dd_sqrt(yz2)));
        dd pre = dd_div(dd_mul(y, dd_sub(dd_mul_d(z2, 3.0), y2)), ddc(6.0));
        out = dd_add(out, dd_mul(pre, a));
    }
    if (xz2.hi > 0.0 && x.hi > 0.0 && y.hi > 0.0) {
        dd a = dd_asinh(dd_div(y, dd_sqrt(xz2)));
        dd pre = dd_div(dd_mul(x, dd_sub(dd_mul_d(z2, 3.0), x2)), ddc(6.0));
        out = dd_add(out, dd_mul(pre, a));
    }
    if (z.hi > 0.0 && x.hi > 0.0 && y.hi > 0.0) {
        dd a = dd_atan(dd_div(dd_mul(x, y), dd_mul(z, R)));
        out = dd_sub(out, dd_mul(dd_div(dd_mul(z, z2), ddc(6.0)), a));
    }
    if (y.hi > 0.0 && x.hi > 0.0 && z.hi > 0.0) {
        dd a = dd_atan(dd_div(dd_mul(x, z), dd_mul(y, R)));
        out = dd_sub(out, dd_mul(dd_mul_d(dd_mul(z, y2), 0.5), a));
    }
    if (x.hi > 0.0 && y.hi > 0.0 && z.hi > 0.0) {
        dd a = dd_atan(dd_div(dd_mul(y, z), dd_mul(x, R)));
        out = dd_sub(out, dd_mul(dd_mul_d(dd_mul(z, x2), 0.5), a));
    }
    return out;
}

// Grid of function c at (i dx, j dy, k dz), 0 <= i <= nx, ... ; stored [k][j][i].
//   c = 0: f(x,y,z)   1: f(y,z,x)   2: f(z,x,y)
//   c = 3: g(x,y,z)   4: g(x,z,y)   5: g(y,z,x)
__global__ void k_newell_fgrid(int c, int gx, int gy, int gz, double dx, double dy, double dz,
                               double2* __restrict__ out) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)gx * gy * gz;
    if (idx >= total) return;
    int i = (int)(idx % gx);
    int j = (int)((idx / gx) % gy);
    int k = (int)(idx / ((long)gx * gy));
    dd x = two_prod((double)i, dx), y = two_prod((double)j, dy), z = two_prod((double)k, dz);
    dd v;
    switch (c) {
        case 0: v = newell_f(x, y, z); break;
        case 1: v = newell_f(y, z, x); break;
        case 2: v = newell_f(z, x, y); break;
        case 3: v = newell_g(x, y, z); break;
        case 4: v = newell_g(x, z, y); break;
        default: v = newell_g(y, z, x); break;
    }
    out[idx] = make_double2(v.hi, v.lo);
}

// parity of function c's grid value under a negative index on each axis
__device__ __forceinline__ int grid_parity(int c, int i, int j, int k) {
    int sx = i < 0 ? -1 : 1, sy = j < 0 ? -1 : 1, sz = k < 0 ? -1 : 1;
    switch (c) {
        case 3: return sx * sy;
        case 4: return sx * sz;
        case 5: return sy * sz;
        default: return 1;
    }
}
// parity of tensor component c under offset sign flips
__device__ __forceinline__ int comp_parity(int c, int sx, int sy, int sz) {
    switch (c) {
        case 3: return sx * sy;
        case 4: return sx * sz;
        case 5: return sy * sz;
        default: return 1;
    }
}

__global__ void k_newell_assemble(int c, int nx, int ny, int nz, int Px, int Py, int Pz,
                                  double dx, double dy, double dz,
                                  const double2* __restrict__ fg, double* __restrict__ grid,
                                  double* __restrict__ octant) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)nx * ny * nz;
    if (idx >= total) return;
    int I = (int)(idx % nx);
    int J = (int)((idx / nx) % ny);
    int K = (int)(idx / ((long)nx * ny));
    const int gx = nx + 1, gy = ny + 1;
    dd acc = ddc(0.0);
    for (int ez = -1; ez <= 1; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
                int i = I + ex, j = J + ey, k = K + ez;
                double w = (ex == 0 ? 2.0 : -1.0) * (ey == 0 ? 2.0 : -1.0) * (ez == 0 ? 2.0 : -1.0);
                w *= (double)grid_parity(c, i, j, k);
                long gi = ((long)abs(k) * gy + abs(j)) * gx + abs(i);
                double2 f = fg[gi];
                acc = dd_add(acc, dd_mul_d(dd{f.x, f.y}, w));
            }
    dd V = dd_mul_d(two_prod(dx, dy), dz);
    dd val = dd_div(acc, dd_mul(dd_mul_d(kPiDD, 4.0), V));
    double v = val.hi + val.lo;
    if (octant) octant[idx] = v;
    for (int sz = -1; sz <= 1; sz += 2) {
        if (sz < 0 && K == 0) continue;
        for (int sy = -1; sy <= 1; sy += 2) {
            if (sy < 0 && J == 0) continue;
            for (int sx = -1; sx <= 1; sx += 2) {
                if (sx < 0 && I == 0) continue;
                int gxi = (sx * I + Px) % Px, gyi = (sy * J + Py) % Py, gzi = (sz * K + Pz) % Pz;
                grid[((long)gzi * Py + gyi) * Px + gxi] = comp_parity(c, sx, sy, sz) * v;
            }
        }
    }
}

bool g_inv_odd_ready[64] = {false};

}  // namespace

int newell_component(mm_ctx* ctx, int c, double* grid, double* octant_out, void* fgrid_scratch) {
    int dev = 0;
    MM_CUDA_CHECK(ctx, cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !g_inv_odd_ready[dev]) {
        init_inv_odd<<<1, 32, 0, ctx->stream>>>();
        MM_LAUNCH_CHECK(ctx);
        g_inv_odd_ready[dev] = true;
    }
    const int gx = ctx->nx + 1, gy = ctx->ny + 1, gz = ctx->nz + 1;
    long gtotal = (long)gx * gy * gz;
    double2* fg = (double2*)fgrid_scratch;
    k_newell_fgrid<<<(unsigned)((gtotal + 127) / 128), 128, 0, ctx->stream>>>(c, gx, gy, gz, ctx->dx, ctx->dy,
                                                                              ctx->dz, fg);
    MM_LAUNCH_CHECK(ctx);
    MM_CUDA_CHECK(ctx, cudaMemsetAsync(grid, 0, sizeof(double) * (size_t)ctx->Px * ctx->Py * ctx->Pz, ctx->stream));
    long total = ctx->N;
    k_newell_assemble<<<(unsigned)((total + 127) / 128), 128, 0, ctx->stream>>>(
        c, ctx->nx, ctx->ny, ctx->nz, ctx->Px, ctx->Py, ctx->Pz, ctx->dx, ctx->dy, ctx->dz, fg, grid, octant_out);
    MM_LAUNCH_CHECK(ctx);
    return MM_OK;
}

}  // namespace mm
