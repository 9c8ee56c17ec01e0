// Blackwell tensor-core helpers (inline PTX): tcgen05 MMA with operands in
// shared memory, accumulators in tensor memory (TMEM), mbarrier completion.
//
// Operand layout used throughout: K-major, no swizzle.  A tile of R rows x K
// elements (16-bit) is stored as 8-row x 16-byte "core matrices" of 128 bytes:
//   byte offset of (row r, element k) = (k / 8) * (R / 8) * 128 + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// so a descriptor has LBO = (R / 8) * 128 (next 8-element K chunk) and
// SBO = 128 (next group of 8 rows); one MMA consumes K = 16 (two chunks) and the
// next MMA starts 2 * LBO further.  8-bit operands use the same byte layout with
// 16 elements per 16-byte chunk (K = 32 per MMA).
#pragma once
#include <cstdint>

namespace cm {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, 16-byte chunk) in a K-major no-swizzle tile of `rows` rows
__device__ __forceinline__ uint32_t chunk_off(int row, int chunk, int rows) {
    return (uint32_t)(chunk * (rows / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
    return d;
}

// Descriptor of a K-major operand tile in the 128-byte swizzle layout: rows of
// 128 bytes, 8-row groups of 1024 bytes (SBO), the 16-byte chunk c of row r
// stored at chunk position c ^ (r % 8).  The tile must start on a 1024-byte
// boundary; a K step inside the 128-byte row is taken by adding its byte offset
// to saddr.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;               // LBO: unused by swizzled K-major layouts
    d |= (uint64_t)(1024 >> 4) << 32;     // SBO: next group of 8 rows
    d |= (uint64_t)1 << 46;               // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;               // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16 with FP32 accumulate; ab = 0 F16, 1 BF16.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int ab) {
    return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4 with FP32 accumulate, both operands E4M3 (format 0).
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_f8f6f4(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_addr(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Waits for the given phase parity; gives up after `limit` polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_addr(mbar)), "r"(parity));
    }
    return done != 0;
}

// One try_wait that may suspend the thread for up to hint_ns nanoseconds while
// the phase is incomplete; it resumes once the phase completes.  A waiting
// thread that sleeps issues no instructions, so the warps it shares an SM
// sub-partition with keep the issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* mbar, uint32_t parity, uint32_t hint_ns) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_addr(mbar)), "r"(parity), "r"(hint_ns) : "memory");
    return done != 0;
}

// Arrival of the issuing thread that also announces `bytes` of bulk copies
// to complete on this barrier (a barrier of count 1 per phase).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(mbar)), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on mbar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int ncols) {  // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_addr(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {  // one full warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;"); }

// TMEM loads.  Each helper issues tcgen05.ld and tcgen05.wait::ld in ONE asm
// statement, so the destination registers are defined only after the wait:
// with separate statements the compiler sees them defined at the load and
// may use them, or spill them to local memory, before the data has arrived.
// Warp w reads lanes 32 (w % 4) .. +31; each thread gets W consecutive FP32
// columns of its lane.
__device__ __forceinline__ void tmem_load16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tmem_load2(uint32_t taddr, uint32_t (&v)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\ntcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]) : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tmem_load4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\ntcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tmem_load8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr) : "memory");
}

// W consecutive columns (W = 2, 4, 8 or 16).
template <int W>
__device__ __forceinline__ void tmem_load(uint32_t taddr, uint32_t (&v)[W]) {
    if constexpr (W == 2) tmem_load2(taddr, v);
    else if constexpr (W == 4) tmem_load4(taddr, v);
    else if constexpr (W == 8) tmem_load8(taddr, v);
    else tmem_load16(taddr, v);
}

}  // namespace tc
}  // namespace cm
