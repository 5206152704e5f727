// mm_energy_noalloc: the energy reduction without a context and without any
// device allocation.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool or arena they do not own, plugins of a host application that hands
// them only its own buffers, or setups where cudaMalloc would synchronise the
// device in the middle of captured or latency-critical work.  This entry
// point serves them: the caller passes m, the demagnetisation field and a
// host array for the result, and the per-block partial sums live in a
// fixed-size array in the library's own device memory (g_energy_scratch,
// 1 MiB, kept by every GPU that loads the library until the process exits).
//
// The array is shared by all calls: calls that overlap on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.  Nothing in it needs clearing: each call overwrites every
// partial sum and result it later reads.
#include <mutex>

#include "mm_internal.cuh"

namespace mm {
namespace {

constexpr int kNoallocThreads = 256;
constexpr long kNoallocMaxBlocks = 32768;
constexpr long kNoallocMaxCells = kNoallocMaxBlocks * kNoallocThreads;   // 8,388,608

// 4 partial sums per block, then the 4 final sums
static __device__ __align__(256) double g_energy_scratch[4 * kNoallocMaxBlocks + 4];

double* g_scratch_addr[64] = {nullptr};
std::mutex g_scratch_mutex;

template <typename T>
__global__ void k_energy_partials(int nx, int ny, int nz, long N, T Ms, T A, T cx, T cy, T cz, double ux, double uy,
                                  double uz, double hx, double hy, double hz, double Ku, double V, double mu0,
                                  const T* __restrict__ m, const T* __restrict__ Hd, double* __restrict__ partial) {
    __shared__ double red[4][kNoallocThreads];
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < N && Ms != (T)0) {
        int x = (int)(i % nx);
        long r = i / nx;
        int y = (int)(r % ny), z = (int)(r / ny);
        T mx = m[i], my = m[i + N], mz = m[i + 2 * N];
        // 6-point exchange field with uniform A (Eq. 2 for unit m)
        T ax = 0, ay = 0, az = 0;
        auto nb = [&](long j, T c) {
            ax += c * (m[j] - mx);
            ay += c * (m[j + N] - my);
            az += c * (m[j + 2 * N] - mz);
        };
        const long sy = nx, sz = (long)nx * ny;
        if (x > 0) nb(i - 1, cx);
        if (x < nx - 1) nb(i + 1, cx);
        if (y > 0) nb(i - sy, cy);
        if (y < ny - 1) nb(i + sy, cy);
        if (z > 0) nb(i - sz, cz);
        if (z < nz - 1) nb(i + sz, cz);
        const double scale = (double)A / (double)Ms;
        double hex = ax * scale, hey = ay * scale, hez = az * scale;
        double ms = (double)Ms;
        e[0] = -0.5 * mu0 * V * ms * ((double)mx * Hd[i] + (double)my * Hd[i + N] + (double)mz * Hd[i + 2 * N]);
        e[1] = -0.5 * mu0 * V * ms * ((double)mx * hex + (double)my * hey + (double)mz * hez);
        double mu = (double)mx * ux + (double)my * uy + (double)mz * uz;
        e[2] = -Ku * V * mu * mu;
        e[3] = -mu0 * V * ms * ((double)mx * hx + (double)my * hy + (double)mz * hz);
    }
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = e[q];
    __syncthreads();
    for (int h = kNoallocThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[4 * (long)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// one block: fixed-order sum of the block partials into out[0..3]
__global__ void k_energy_final(const double* __restrict__ partial, long nblocks, double* __restrict__ out) {
    __shared__ double red[4][kNoallocThreads];
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    for (long b = threadIdx.x; b < nblocks; b += kNoallocThreads)
        for (int q = 0; q < 4; ++q) e[q] += partial[4 * b + q];
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = e[q];
    __syncthreads();
    for (int h = kNoallocThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

// Device address of g_energy_scratch on `dev`, looked up once per device
// with that device current.
int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= 64) return fail(nullptr, MM_ERR_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return fail(nullptr, MM_ERR_CUDA, "cudaGetSymbolAddress of the energy scratch failed: %s",
                        cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return MM_OK;
}

template <typename T>
int run(int nx, int ny, int nz, double dx, double dy, double dz, double Ms, double A, double Ku, const double u[3],
        const double h[3], const void* m, const void* Hd, double* E_out, cudaStream_t stream, double* scratch) {
    const long N = (long)nx * ny * nz;
    const long nblocks = (N + kNoallocThreads - 1) / kNoallocThreads;
    const T cx = (T)(2.0 / (kMu0 * dx * dx)), cy = (T)(2.0 / (kMu0 * dy * dy)), cz = (T)(2.0 / (kMu0 * dz * dz));
    k_energy_partials<T><<<(unsigned)nblocks, kNoallocThreads, 0, stream>>>(
        nx, ny, nz, N, (T)Ms, (T)A, cx, cy, cz, u[0], u[1], u[2], h[0], h[1], h[2], Ku, dx * dy * dz, kMu0,
        (const T*)m, (const T*)Hd, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_energy_final<<<1, kNoallocThreads, 0, stream>>>(scratch, nblocks, scratch + 4 * kNoallocMaxBlocks);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E_out, scratch + 4 * kNoallocMaxBlocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(nullptr, MM_ERR_CUDA, "mm_energy_noalloc: %s", cudaGetErrorString(e));
    return MM_OK;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" int mm_energy_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, int precision, double Ms,
                                 double A, double Ku, const double u_anis[3], const double h_ext[3], const void* m,
                                 const void* H_demag, double E_out[4], void* stream) {
    if (nx < 1 || ny < 1 || nz < 1)
        return fail(nullptr, MM_ERR_INVALID_ARG, "mm_energy_noalloc: mesh sizes must be >= 1");
    const long N = (long)nx * ny * nz;
    if (N > kNoallocMaxCells)
        return fail(nullptr, MM_ERR_INVALID_ARG,
                    "mm_energy_noalloc: %ld cells exceed the fixed scratch of this entry point (at most %ld cells); "
                    "use mm_energy with a context instead",
                    N, kNoallocMaxCells);
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return fail(nullptr, MM_ERR_INVALID_ARG, "mm_energy_noalloc: cell size must be finite and > 0");
    if (precision != MM_F32 && precision != MM_F64)
        return fail(nullptr, MM_ERR_INVALID_ARG, "mm_energy_noalloc: bad precision");
    if (!(Ms >= 0) || !(A >= 0) || !std::isfinite(Ms) || !std::isfinite(A) || !std::isfinite(Ku))
        return fail(nullptr, MM_ERR_INVALID_ARG, "mm_energy_noalloc: Ms, A must be finite and >= 0");
    if (!m || !H_demag || !E_out) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_energy_noalloc: null pointer");
    double u[3] = {0.0, 0.0, 1.0};
    if (u_anis) {
        double n = std::sqrt(u_anis[0] * u_anis[0] + u_anis[1] * u_anis[1] + u_anis[2] * u_anis[2]);
        if (!(n > 0) || !std::isfinite(n)) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_energy_noalloc: zero axis");
        for (int c = 0; c < 3; ++c) u[c] = u_anis[c] / n;
    }
    double h[3] = {0.0, 0.0, 0.0};
    if (h_ext)
        for (int c = 0; c < 3; ++c) h[c] = h_ext[c];
    cudaStream_t st = (cudaStream_t)stream;
    int caller_dev = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&caller_dev);
    if (e == cudaSuccess) {
        dev = caller_dev;
        if (st) e = cudaStreamGetDevice(st, &dev);
    }
    if (e == cudaSuccess && dev != caller_dev) e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MM_ERR_CUDA, "mm_energy_noalloc: cannot select the stream's device: %s",
                    cudaGetErrorString(e));
    }
    // the stream's device is current for the call; the caller's current
    // device is put back on every return path
    struct RestoreDevice {
        int dev;
        bool on;
        ~RestoreDevice() {
            if (on) cudaSetDevice(dev);
        }
    } restore{caller_dev, dev != caller_dev};
    double* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    if (precision == MM_F64) return run<double>(nx, ny, nz, dx, dy, dz, Ms, A, Ku, u, h, m, H_demag, E_out, st, scratch);
    return run<float>(nx, ny, nz, dx, dy, dz, Ms, A, Ku, u, h, m, H_demag, E_out, st, scratch);
}
