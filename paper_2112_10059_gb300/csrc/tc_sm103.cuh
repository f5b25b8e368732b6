// Blackwell (sm_100 family) tensor-core primitives as inline PTX: shared-memory
// matrix descriptors, tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in TMEM),
// TMEM allocation and loads, mbarriers with bounded waits, and bulk async copies.
//
// Operand layout used throughout: K-major, 128-byte swizzle.  A [rows][K] BF16
// tile is stored as K/64 chunks; chunk c holds rows x 64 elements, row r at byte
// r*128, and the 16-byte unit u of a row at ((u ^ (r & 7)) * 16).  Chunks and
// the 8-row groups inside them (1024 bytes) are 1024-byte aligned.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) of a K-major SW128 BF16 tile with `rows` rows
__host__ __device__ __forceinline__ uint32_t sw128_offset(int r, int k, int rows) {
    int chunk = k >> 6, kk = k & 63;
    int unit = kk >> 3, within = (kk & 7) * 2;
    return (uint32_t)(chunk * rows * 128 + r * 128 + ((unit ^ (r & 7)) << 4) + within);
}

// Shared-memory matrix descriptor (sm_100 format): start address >> 4 in [0,14),
// leading byte offset >> 4 in [16,30), stride byte offset >> 4 in [32,46),
// descriptor version 1 in [46,48), layout type in [61,64) (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                    // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;          // SBO: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                    // version
    d |= (uint64_t)2u << 61;                    // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ __forceinline__ uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar_saddr) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_saddr)
                 : "memory");
}

// TMEM allocation by one full warp; the base address is written to shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_saddr, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_saddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy writes to shared memory -> visible to the async proxy (tensor core reads)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 16 columns of 32-bit TMEM data per warp (lane = row of D).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t saddr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t saddr, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t saddr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(saddr), "r"(parity)
        : "memory");
    return ok;
}
// Bounded wait: returns false after max_iter unsuccessful polls (the caller records an error).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t saddr, uint32_t parity, uint32_t max_iter) {
    for (uint32_t i = 0; i < max_iter; ++i)
        if (mbar_try_wait(saddr, parity)) return true;
    return false;
}

// 1D bulk async copy global -> shared, completion counted on an mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(uint32_t dst_saddr, const void *src, uint32_t bytes, uint32_t mbar_saddr) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst_saddr),
                 "l"(src), "r"(bytes), "r"(mbar_saddr)
                 : "memory");
}

// Bulk reduction shared -> global: dst[0..bytes/4) += src[0..bytes/4) (FP32 adds performed at
// the L2, one request per line instead of one per warp-wide 32-float segment); both addresses
// 16-byte aligned, bytes a multiple of 16.  Tracked by the issuing thread's bulk group.
__device__ __forceinline__ void bulk_reduce_add_f32(float *dst, uint32_t src_saddr, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst),
                 "r"(src_saddr), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// until the source shared memory of every committed bulk operation of this thread has been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (generic proxy); src_bytes = 0 writes zeros and
// reads nothing.  Completion is tracked per thread with commit / wait groups.
__device__ __forceinline__ void cp_async16(uint32_t dst_saddr, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst_saddr), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// FP32 -> BF16, round to nearest even
__device__ __forceinline__ uint16_t f2bf(float x) {
    uint32_t u = __float_as_uint(x);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// split an FP32 value into BF16 hi + lo (x ~ hi + lo to ~16 bits)
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
    uint32_t u = __float_as_uint(x);
    // round to nearest even on the top 16 bits
    uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);
    hi = (uint16_t)(r >> 16);
    float h = __uint_as_float((uint32_t)hi << 16);
    float d = x - h;
    uint32_t v = __float_as_uint(d);
    uint32_t s = v + 0x7FFFu + ((v >> 16) & 1u);
    lo = (uint16_t)(s >> 16);
}

}  // namespace tc
}  // namespace sph
