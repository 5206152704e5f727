// Tensor Memory Accelerator (TMA) building blocks of the TMA-fed demag
// passes, written from the PTX ISA's descriptions of cp.async.bulk.tensor and
// the mbarrier transaction count.
//
// A tile copy is described by a tensor map (CUtensorMap, encoded on the host
// by the driver's cuTensorMapEncodeTiled, which the library looks up through
// the runtime so it does not link libcuda).  One thread arms an mbarrier with
// the byte count it expects (arrive.expect_tx) and issues the copies; each
// copy's completion subtracts its bytes, and the phase flips when all have
// landed.  Waiting threads poll the phase with a bounded loop.
// Alignment rules kept by every caller: the innermost coordinate times the
// element size is a multiple of 16 bytes, the global base is 16-byte aligned
// and the global strides are multiples of 16 bytes (the encoder checks the
// last two), and each shared-memory destination is 128-byte aligned.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "mm_tcgen05.cuh"

namespace mm {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// this thread's arrival, and `bytes` more expected before the phase completes
__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// make the mbarrier initialisation visible to the copy engine
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this block's earlier generic-proxy accesses of shared memory before a
// following copy into it (async proxy)
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// box of a 3-D tensor map at coordinates (c0 innermost, c1, c2) into shared
// memory at dst, completing `bytes of the box` on mbar
__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

// `bytes` contiguous bytes (a multiple of 16, both addresses 16-byte
// aligned) from global memory into shared memory at dst, completing on mbar
__device__ __forceinline__ void load_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

}  // namespace tma

// Host: encode a 3-D FP32 tensor map over dims (d0 innermost, d1, d2) with
// byte strides s1, s2 and box (b0, b1, b2), no swizzle, zero fill.  Returns
// false when the driver has no encoder or rejects the description.
bool tma_encode_3d(void* map128, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1, uint64_t s2,
                   uint32_t b0, uint32_t b1, uint32_t b2);

}  // namespace mm
