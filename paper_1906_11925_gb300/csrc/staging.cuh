// Bulk asynchronous global -> shared copies completing on an mbarrier, and
// bounded mbarrier waits (the staging of the table-staged kernels).  Every
// wait polls at most `limit` times; the caller turns a give-up into an error
// flag and returns, so no kernel can hang on a copy that never lands.
#pragma once

#include <cstdint>

namespace hemelb_gb300 {
namespace {

constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity,
                                                  unsigned limit = kWaitLimit) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk prefetch of `bytes` bytes at p into L2 (no destination, no barrier:
// the copy engine fetches the lines while the issuing thread goes on).  p
// must be 16-byte aligned, bytes a multiple of 16, and the whole range inside
// one allocation.
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The bulk AA step kernels prefetch into L2, at their start, the rows of the
// tile HGB_PF_BLOCKS blocks ahead of their own (the blocks of a launch start
// roughly in index order, so that tile is read a few block lifetimes later):
// more bytes in flight per SM than the threads' own loads give at the
// occupancy their registers allow.  0 switches it off.  (The AA adjoint
// kernels do the same with their own distances.)
#ifndef HGB_PF_BLOCKS
#define HGB_PF_BLOCKS 608
#endif

// The prefetch of one tile: nrows rows of `elem` bytes per site, row r at
// base + r * row_stride elements, sites [x0, x0 + 256) clipped to the row
// length npad (a multiple of 128, so every range stays 256-byte aligned and
// a multiple of 16 bytes); thread r in [0, nrows) issues row r.  Returns at
// once when x0 is at or past `limit`.
__device__ __forceinline__ void prefetch_rows(const void *base, unsigned elem, unsigned row_stride, int nrows,
                                              unsigned x0, unsigned limit, unsigned npad, int r) {
    if (r < 0 || r >= nrows || x0 >= limit) return;
    const unsigned cnt = min(256u, npad - x0);
    const char *p = (const char *)base + ((size_t)r * row_stride + x0) * elem;
    l2_prefetch(p, cnt * elem);
}

}  // namespace
}  // namespace hemelb_gb300
