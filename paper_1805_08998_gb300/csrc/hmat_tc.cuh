// hmat_tc.cuh -- fifth-generation tensor-core building blocks for sm_103a, in inline PTX:
// tensor-memory (TMEM) allocation, shared-memory descriptors of K-major operands without
// swizzling, kind::tf32 MMAs with an FP32 accumulator in TMEM, commits to an mbarrier with
// bounded waits, and TMEM loads.
//
// Operand layout (no swizzle, K-major): the operand is cut into core matrices of 8 rows x 16 bytes
// (8 rows x 4 TF32 values, 128 contiguous bytes, row r at byte 16 r). The descriptor's leading
// byte offset (LBO) is the distance between core matrices adjacent along K, its stride byte
// offset (SBO) the distance between groups of 8 rows. An MMA of K = 8 reads two core matrices
// along K per group of 8 rows.
//
// Accumulator layout in TMEM (cta_group::1): with M = 64, rows 16 q .. 16 q + 15 sit in lanes
// 32 q .. 32 q + 15 (q = 0..3); with M = 128, row i sits in lane i. Column j of the result is the
// j-th 32-bit column after the accumulator's base column. A warp reads lanes 32 (warp % 4) ..
// 32 (warp % 4) + 31 only.
#pragma once
#include <cstdint>

namespace hm {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// descriptor of a K-major operand without swizzling that starts at shared address addr
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 operands, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) (+)= A B^T over K = 8; issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive once on mbar when every MMA issued so far by this thread has completed
__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

// wait for the phase with the given parity of mbar to complete, giving up after `limit` polls;
// true when it completed
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; it++)
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory writes of this thread made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// warp-collective: allocate ncols (a power of two >= 32) TMEM columns, base address to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// warp-collective
__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// warp-collective: 16 consecutive 32-bit columns from taddr of the warp's 32 lanes (one lane per
// thread), then wait for the load
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; c++) v[c] = __uint_as_float(r[c]);
}

// x rounded to TF32 (nearest, ties away from zero): an FP32 value whose low 13 mantissa bits are
// zero. x = hi + (x - hi) exactly, and the remainder carries the next 11 bits when it is itself
// read as TF32, so three TF32 products (hi hi, hi lo, lo hi) give a product to about FP32 accuracy.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace hm
