// Thin inline-PTX layer over the sm_100/sm_103 tensor-core path: tensor memory
// (TMEM) allocation, tcgen05.mma of kind::tf32 with FP32 accumulation,
// completion through an mbarrier, TMEM -> register loads, and bulk
// global -> shared copies (TMA engine) that complete on the same mbarriers.
//
// Operand layout (both operands K-major, no swizzle): an operand of R rows
// (the M or N extent) and Kt columns (K) of 4-byte elements is stored as 8 x 4
// "core matrices" of 128 contiguous bytes (row i of a core matrix at +16 i):
//   byte(row, k) = (row / 8) * SBO + (k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4,
//   SBO = Kt * 32 (the K-adjacent core matrices of one 8-row group are
//   consecutive, LBO = 128).
// One instruction consumes K = 8 (two core matrices along K); the operand of
// the instruction at K offset k0 starts k0 * 32 bytes into the buffer.
//
// Every wait here is bounded: a wait that runs past its cycle budget returns
// false and the caller raises its flag instead of spinning forever.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gpeps {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) in the K-major no-swizzle operand layout
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int Kt) {
  return (uint32_t)((row >> 3) * (Kt * 32) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K direction), stride byte offset (8-row groups), the fixed version
// field of sm_100 (bit 46), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in FP32, A and B in TF32, both
// K-major, M x N tile (M = 128: TMEM lane m holds row m).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------- TMEM
// Allocation by one whole warp; the address is written to *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
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
// generic-proxy writes to shared memory -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// generic-proxy accesses of global and shared memory ordered before later async-proxy ones
// (bulk copies reading tensors that generic stores wrote, into shared memory generic code used)
__device__ __forceinline__ void fence_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// ---------------------------------------------------------------- MMA
// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on the mbarrier when every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes (this warp's quarter of TMEM) x 32 consecutive FP32 columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 16 consecutive FP32 columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised mbarriers visible to the async proxy (bulk copies, MMA commits)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete, for at most `limit` SM
// cycles; false if it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// ---------------------------------------------------------------- bulk copy (TMA engine)
// bytes from global to shared (both 16-byte aligned, bytes a multiple of 16),
// completing as transaction bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// FP32 -> (hi, lo) with hi = x rounded to TF32 (10 stored mantissa bits) and
// lo = x - hi (exact in FP32) rounded to TF32, so that x y is
// hi_x hi_y + hi_x lo_y + lo_x hi_y to about 2^-22 |x y| (the 3xTF32 split).
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

}  // namespace tc

// ---------------------------------------------------------------- shared pieces of the tensor-core passes
struct TcCtx {
  uint32_t tmem;    // TMEM base address (tc_cols(D) columns)
  uint64_t* bar;    // mbarrier the MMA commits arrive on
  uint64_t* sbar;   // mbarrier of the bulk-copy staging
  long long limit;  // wait budget in SM cycles
};

__device__ __forceinline__ void tc_put(unsigned char* hi, unsigned char* lo, int row, int q, int Kt, float x) {
  float h, l;
  tc::split_tf32(x, h, l);
  const uint32_t o = tc::kmajor_off(row, q, Kt);
  *reinterpret_cast<float*>(hi + o) = h;
  *reinterpret_cast<float*>(lo + o) = l;
}

// Every thread waits for a phase of the mbarrier; the outcome is made uniform
// over the CTA.  After a wait that gave up, a second bounded wait lets the
// operations still in flight finish before the caller reuses the memory.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t& phase, long long limit) {
  const bool ok = __syncthreads_and(tc::mbar_wait(bar, phase, limit) ? 1 : 0) != 0;
  if (!ok) tc::mbar_wait(bar, phase, limit);
  phase ^= 1u;
  return ok;
}

// Thread 0: the 3xTF32 products of `nk` K values (a multiple of 8) of the
// staged operands.  a/b: shared addresses of hi (lo at +lo_a / +lo_b bytes);
// Kt: K extent of the operand layout.
__device__ __forceinline__ void tc_issue(uint32_t a, uint32_t lo_a, uint32_t b, uint32_t lo_b, int nk, int Kt,
                                         uint32_t d_tmem, uint32_t idesc, bool fresh) {
  const uint32_t lbo = 128, sbo = (uint32_t)Kt * 32;
  for (int ks = 0; ks < nk; ks += 8) {
    const uint32_t off = (uint32_t)ks * 32;
    const uint64_t ah = tc::smem_desc(a + off, lbo, sbo), al = tc::smem_desc(a + lo_a + off, lbo, sbo);
    const uint64_t bh = tc::smem_desc(b + off, lbo, sbo), bl = tc::smem_desc(b + lo_b + off, lbo, sbo);
    tc::mma_tf32(d_tmem, ah, bh, idesc, (fresh && ks == 0) ? 0u : 1u);
    tc::mma_tf32(d_tmem, ah, bl, idesc, 1u);
    tc::mma_tf32(d_tmem, al, bh, idesc, 1u);
  }
}

}  // namespace gpeps
