// Fifth-generation tensor core (tcgen05) building blocks for sm_103a, in
// inline PTX (PTX ISA: tcgen05.alloc / mma / commit / ld / fence, mbarrier):
// tensor-memory allocation, shared-memory matrix descriptors of the
// K-major canonical layout without swizzle, the instruction descriptor of
// kind::tf32 with FP32 accumulation, one-thread MMA issue with completion
// counted on an mbarrier, and warp loads of the accumulator.
//
// Operand layout (K-major, no swizzle): a plane of R rows x KC columns of
// 32-bit elements is a grid of core matrices of 8 rows x 4 elements (8 x 16
// bytes, 128 contiguous bytes, row r at byte 16 r); core (r / 8, k / 4)
// starts at (r / 8) * SBO + (k / 4) * LBO with LBO = 128 bytes (cores
// adjacent along K contiguous) and SBO = (KC / 4) * 128 bytes.  One MMA of
// kind::tf32 consumes K = 8 columns (two cores along K); the next K step
// starts 2 * LBO = 256 bytes further.
#pragma once

#include <cstdint>

namespace gcq {
namespace tc {

constexpr uint32_t kLBO = 128;   // bytes between K-adjacent core matrices

__host__ __device__ constexpr uint32_t sbo_bytes(int kc) { return (uint32_t)(kc / 4) * 128u; }
// byte offset of element (r, k) in a plane with KC columns
__host__ __device__ constexpr uint32_t plane_off(int r, int k, int kc) {
  return (uint32_t)(r >> 3) * sbo_bytes(kc) + (uint32_t)(k >> 2) * kLBO + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address >> 4 in bits 0-13, leading
// dimension byte offset >> 4 in bits 16-29, stride dimension byte offset >> 4
// in bits 32-45, the fixed value 1 in bits 46-48, base offset 0, relative
// leading-dimension mode, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::tf32: D in FP32 (bits 4-5 = 1),
// A and B in TF32 (bits 7-9 and 10-12 = 2), no negation, both operands
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] = A B^T (+ D if acc): one MMA, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// the mbarrier receives one arrival when every MMA issued so far by this
// thread has completed
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// tensor-memory allocation of ncols columns (power of two >= 32) by one whole
// warp; the base address is written to *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane (the warp
// reads lanes 32 (warp % 4) .. + 31; taddr carries that lane base)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// round to the nearest TF32 value (10 explicit mantissa bits; NaN and
// infinities kept)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi): the split whose three
// products hi hi + hi lo + lo hi carry about 21 bits of each FP32 product
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - hi);
}

}  // namespace tc
}  // namespace gcq
