// Fifth-generation tensor cores (tcgen05) from inline PTX: tensor-memory
// allocation, shared-memory matrix descriptors, the BF16 MMA with an FP32
// accumulator in tensor memory, its completion on an mbarrier, and the
// read-back of the accumulator into registers.
//
// Operands sit in shared memory in the no-swizzle K-major layout: an operand
// of R rows (M or N) and K columns is cut into core matrices of 8 rows x 16
// bytes (8 BF16 values of K), each 128 contiguous bytes with row r at byte
// 16 r.  A descriptor gives the start address, the byte distance between
// core matrices that are neighbours along K (the leading-dimension offset)
// and between neighbours along M/N (the stride-dimension offset).  The
// layouts used here put the 8-row groups of one K-group next to each other
// (stride 128 bytes) and the K-groups R * 16 bytes apart, so element (r, k)
// of an operand lives at byte (k / 8) R 16 + (r / 8) 128 + (r % 8) 16 + (k % 8) 2.
#pragma once
#include <stdint.h>

namespace cbp {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of an R-row operand in the layout above.
__host__ __device__ constexpr uint32_t kmajor_offset(int R, int r, int k) {
  return (uint32_t)((k >> 3) * R * 16 + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (no swizzle): start address, leading- and
// stride-dimension byte offsets in 16-byte units, the descriptor version
// (bits 46-48 = 0b001) and swizzle mode 0 in bits 61-63.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both
// operands K-major, dense: D format in bits 4-5, A and B formats in bits 7-9
// and 10-12, N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The encodings, checked at compile time: the shapes of the library's MMAs
// (M = 128; N = 32 and 16) and the operand layout's neighbours.
static_assert(idesc_bf16_f32(128, 32) == 0x08080490u, "kind::f16 descriptor, BF16 x BF16 -> F32, 128 x 32");
static_assert(idesc_bf16_f32(128, 16) == 0x08040490u, "kind::f16 descriptor, BF16 x BF16 -> F32, 128 x 16");
static_assert(kmajor_offset(128, 1, 0) == 16 && kmajor_offset(128, 8, 0) == 128 &&
                  kmajor_offset(128, 0, 1) == 2 && kmajor_offset(128, 0, 8) == 128 * 16,
              "rows 16 bytes apart in a core matrix, 8-row groups 128 bytes apart, K-groups R * 16");

// Tensor memory: `ncols` columns (a power of two, >= 32) for this CTA, by one
// whole warp; the base address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor core's reads.
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D (tensor memory) = A B^T (+ D when `accumulate`), one 128 x N x 16 step.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
// The mbarrier's phase completes once every MMA this thread issued before has.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   saddr(bar))
               : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Wait for phase `parity`, giving up after `limit` polls.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, int limit) {
  const uint32_t a = saddr(bar);
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of the accumulator rows this warp may read
// (lanes 32 (warp % 4) .. + 31; thread i gets row 32 (warp % 4) + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr)
      : "memory");
  // the registers pass through the wait, so no use of them is scheduled before it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
                 "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace tc
}  // namespace cbp
