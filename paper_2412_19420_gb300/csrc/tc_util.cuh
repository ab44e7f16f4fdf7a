// tc_util.cuh -- device helpers shared by the tcgen05 pair passes: mbarriers
// with bounded waits, cp.async staging, the SWIZZLE_128B shared-memory and
// kind::f8f6f4 instruction descriptors, MMA issue and commit, and the
// bit -> e4m3 expansion of 0/1 operands.
#pragma once

#include "fim_common.cuh"

namespace fim_tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and *abort set) when wait_ns of %globaltimer pass, or
// when another role of the CTA has already set *abort.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity, int *abort,
                                                  unsigned long long wait_ns) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t i = 1;; i++) {
        if (mbar_try(b, parity)) return true;
        if ((i & 63) == 0) {
            if (*(volatile int *)abort) return false;
            if (globaltimer_ns() - t0 > wait_ns) {
                atomicExch(abort, 1);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4)  // start address
           | (1ull << 16)                        // leading byte offset (unused for swizzled K-major)
           | ((uint64_t)(1024 >> 4) << 32)       // stride byte offset
           | (1ull << 46)                        // descriptor version
           | (2ull << 61);                       // SWIZZLE_128B
}

// Instruction descriptor: kind::f8f6f4, A = B = E4M3, D = F32, K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f8(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// A from tensor memory (row m in lane m, K bytes packed 4 per 32-bit column).
__device__ __forceinline__ void mma_f8_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 4 bits -> 4 bytes of e4m3 (0x40 = 2.0, 0x00 = 0.0), bit j -> byte j.
// x * 0x08102040 is x << 6 + x << 13 + x << 20 + x << 27: the four copies
// occupy bits 6-9, 13-16, 20-23, 27-30 (no carries), and bit j of the copy
// shifted by 6 + 7j lands on bit 8j + 6, the only set bit of 0x40 in byte j.
// A set bit is encoded as 2.0 (one bit, two instructions per 4 bytes); every
// product is then 4, so the epilogue divides the exact sums by 4.
__device__ __forceinline__ uint32_t nib_to_e4m3(uint32_t x) {
    return (x * 0x08102040u) & 0x40404040u;
}
__device__ __forceinline__ uint4 bits16_to_e4m3(uint32_t h) {
    return make_uint4(nib_to_e4m3(h & 15u), nib_to_e4m3((h >> 4) & 15u), nib_to_e4m3((h >> 8) & 15u),
                      nib_to_e4m3((h >> 12) & 15u));
}

// Row r of a SWIZZLE_128B K-major tile (128 bytes per row): 16-byte chunk c
// lives at (r / 8) * 1024 + (r % 8) * 128 + ((c ^ (r % 8)) * 16).
__device__ __forceinline__ void store_row(uint8_t *tile, int r, uint4 w) {
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    uint8_t *row = tile + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const uint32_t h = (words[c >> 1] >> ((c & 1) * 16)) & 0xFFFFu;
        *reinterpret_cast<uint4 *>(row + ((c ^ (r & 7)) << 4)) = bits16_to_e4m3(h);
    }
}

// Row of A (this thread's TMEM lane) at columns [col, col + 32): word t of
// the 128-byte row holds K elements 4t .. 4t + 3.
__device__ __forceinline__ void store_row_tmem(uint32_t taddr, uint4 w) {
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; q++) {  // 32 bits = 32 elements = 8 columns per store
        uint32_t v[8];
        const uint4 lo = bits16_to_e4m3(words[q] & 0xFFFFu), hi = bits16_to_e4m3(words[q] >> 16);
        v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
        v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
        tmem_st8(taddr + 8u * q, v);
    }
}

// Row r of a SWIZZLE_128B K-major tile (128 bytes per row) filled with zeros.
__device__ __forceinline__ void zero_row(uint8_t *tile, int r) {
    uint8_t *row = tile + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
    for (int c = 0; c < 8; c++) *reinterpret_cast<uint4 *>(row + (c << 4)) = make_uint4(0, 0, 0, 0);
}

}  // namespace fim_tc
