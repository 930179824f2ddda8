// Tensor memory (TMEM) as per-thread accumulator storage (sm_100 family).
//
// TMEM is the 256 KB per SM (128 lanes x 512 columns of 32 bits) that the
// fifth-generation tensor cores accumulate into.  The backward kernel uses it
// without the tensor cores: it holds spectra that must survive a whole tile
// but do not fit in registers (the per-(source, microphone) correlation
// accumulators of the RIR gradient).  A warp may only touch the 32 lanes of
// its quadrant (warp index mod 4); each thread owns one lane and a run of
// columns, so no data ever moves between threads through TMEM and no
// cross-thread ordering is needed beyond the allocation itself.
//
// Every load is fused with its wait (tcgen05.wait::ld) and every store with
// its wait (tcgen05.wait::st) in one asm statement: the loaded registers are
// then defined when the statement ends, so the compiler cannot schedule a use
// before the data has landed, and a later load of the same columns always
// sees the store.
#pragma once
#include <stdint.h>

#include "rsim_fft.cuh"

namespace rsim {

// Allocates ncols columns (a power of two, 32 .. 512) for the CTA and writes
// the base address to *dst (shared memory).  Executed by one whole warp.
// Blocks until the columns are free (another CTA on the SM may hold them).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
// After the allocation: this CTA will not allocate again (lets a waiting CTA
// on the same SM proceed as soon as columns are freed).  One whole warp.
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
// Frees the CTA's columns.  One whole warp; every thread's TMEM accesses must
// be complete and ordered before it (tmem_fence_before, barrier, tmem_fence_after).
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// v[0 .. 2E) <- 2E consecutive columns of this thread's lane (warp-collective:
// every thread of the warp passes the same address, the quadrant's base lane).
template <int E>
__device__ __forceinline__ void tmem_load(float2 (&v)[E], uint32_t taddr);
template <int E>
__device__ __forceinline__ void tmem_store(uint32_t taddr, const float2 (&v)[E]);

#define RSIM_R8(a, o) "=r"(a[o + 0]), "=r"(a[o + 1]), "=r"(a[o + 2]), "=r"(a[o + 3]), "=r"(a[o + 4]), \
                      "=r"(a[o + 5]), "=r"(a[o + 6]), "=r"(a[o + 7])
#define RSIM_W8(a, o) "r"(a[o + 0]), "r"(a[o + 1]), "r"(a[o + 2]), "r"(a[o + 3]), "r"(a[o + 4]), \
                      "r"(a[o + 5]), "r"(a[o + 6]), "r"(a[o + 7])

template <>
__device__ __forceinline__ void tmem_load<8>(float2 (&v)[8], uint32_t taddr) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : RSIM_R8(r, 0), RSIM_R8(r, 8)
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
}

template <>
__device__ __forceinline__ void tmem_store<8>(uint32_t taddr, const float2 (&v)[8]) {
    uint32_t r[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        r[2 * e] = __float_as_uint(v[e].x);
        r[2 * e + 1] = __float_as_uint(v[e].y);
    }
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n"
        "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
        RSIM_W8(r, 0), RSIM_W8(r, 8)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_load<16>(float2 (&v)[16], uint32_t taddr) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : RSIM_R8(r, 0), RSIM_R8(r, 8), RSIM_R8(r, 16), RSIM_R8(r, 24)
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
}

template <>
__device__ __forceinline__ void tmem_store<16>(uint32_t taddr, const float2 (&v)[16]) {
    uint32_t r[32];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        r[2 * e] = __float_as_uint(v[e].x);
        r[2 * e + 1] = __float_as_uint(v[e].y);
    }
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n"
        "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
        RSIM_W8(r, 0), RSIM_W8(r, 8), RSIM_W8(r, 16), RSIM_W8(r, 24)
        : "memory");
}

#undef RSIM_R8
#undef RSIM_W8

// TMEM address of this thread's accumulator columns: the lanes of its warp's
// quadrant, and for warps beyond the first four the next run of 2E columns.
// T threads own T / 128 such runs per accumulator (kWCols columns in all).
template <int E>
__device__ __forceinline__ uint32_t tmem_thread_addr(uint32_t base, int t) {
    const int w = t >> 5;
    return base + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((w >> 2) * 2 * E);
}

}  // namespace rsim
