// Inline-PTX helpers for the 5th-generation tensor cores of sm_103a:
// tensor-memory allocation, tcgen05.mma with shared-memory descriptors,
// commits to mbarriers, tensor-memory loads and 2D TMA tile loads.
#pragma once

#include <stdint.h>

#include "ptx.cuh"

namespace grom {
namespace tc {

// ---------------------------------------------------------------- TMEM
// Allocates `ncols` (power of two >= 32) columns of tensor memory for this
// CTA; the base address is written to *dst (shared memory).  Whole warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_addr(dst)),
               "r"(ncols)
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

// ------------------------------------------------------------- descriptors
// Shared-memory matrix descriptor for a K-major operand stored in the
// 128-byte swizzled canonical layout: rows of 128 bytes (64 bf16 along K),
// 8-row atoms of 1024 bytes stacked along M/N (stride byte offset 1024).
// The tile base must be 1024-byte aligned; advancing along K inside the
// 128-byte span is done by adding bytes/16 to the start-address field.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(const void* smem_tile) {
  const uint64_t addr = (uint64_t)(ptx::smem_addr(smem_tile) >> 4) & 0x3FFFull;
  const uint64_t lbo = 1ull;              // unused for swizzled K-major; conventional 16 B
  const uint64_t sbo = 1024ull >> 4;      // 8 rows x 128 B
  return addr | (lbo << 16) | (sbo << 32) | (1ull << 46) /* descriptor version */ | (2ull << 61) /* SWIZZLE_128B */;
}

// Shared-memory matrix descriptor for an MN-major operand in the 128-byte
// swizzled canonical layout: rows of 128 bytes hold 64 bf16 along M (or N),
// consecutive rows are consecutive K, 8-row atoms of 1024 bytes.  `sbo` is the
// byte offset between atoms along K (8 rows further), `lbo` the byte offset
// between 64-element blocks along M.  Advancing K by 16 adds 2 atoms
// (2 * sbo bytes) to the start address.
__device__ __forceinline__ uint64_t sw128_mnmajor_desc(const void* smem_tile, uint32_t lbo, uint32_t sbo) {
  const uint64_t addr = (uint64_t)(ptx::smem_addr(smem_tile) >> 4) & 0x3FFFull;
  return addr | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both operands
// K-major, dense, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                         // D format: F32
         | (1u << 7)                       // A format: BF16
         | (1u << 10)                      // B format: BF16
         | ((uint32_t)(N >> 3) << 17)      // N / 8
         | ((uint32_t)(M >> 4) << 24);     // M / 16
}

// The same with A MN-major (the "transpose A" bit) and B K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32_amn(int M, int N) {
  return idesc_bf16_f32(M, N) | (1u << 15);
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on an mbarrier once all previously issued tcgen05.mma of this
// thread have completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   ptx::smem_addr(bar))
               : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp receives
// lane (base lane + t), columns col .. col+31.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// 2D tiled load of box (x = inner coordinate, y = row) into shared memory,
// completing on an mbarrier.  x * element size must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int32_t x, int32_t y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(ptx::smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(ptx::smem_addr(bar))
      : "memory");
}

// 3D tiled load of box (x, y, z) into shared memory, completing on an
// mbarrier.  x * element size must be a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int32_t x, int32_t y, int32_t z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(ptx::smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(ptx::smem_addr(bar))
      : "memory");
}

}  // namespace tc
}  // namespace grom
