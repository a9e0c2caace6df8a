// Blackwell (sm_103a) building blocks written as inline PTX: mbarriers,
// TMA tile loads, tensor-memory allocation, tcgen05 MMA / commit / load and
// the shared-memory matrix descriptors they consume.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

__device__ __forceinline__ uint32_t hpc_smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier -------------------------------------------------------------
__device__ __forceinline__ void hpc_mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(hpc_smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void hpc_mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(hpc_smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void hpc_mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(hpc_smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool hpc_mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(hpc_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As hpc_mbar_try_wait, but a thread whose phase is not complete yet is
// suspended (up to hint_ns) until it is, instead of returning at once: the
// waiting warp takes no issue slots from the others.
__device__ __forceinline__ bool hpc_mbar_try_wait_sleep(uint64_t *bar, uint32_t parity,
                                                        uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(hpc_smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Waits for the completion of the phase with the given parity.  Gives up
// (returns false) when *abort is set by another role, or after limit_ns, in
// which case it records HPC_ERR_TIMEOUT and sets *abort.
__device__ __forceinline__ bool hpc_mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort,
                                              int *status, uint64_t limit_ns) {
  if (hpc_mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = hpc_globaltimer();
  for (uint32_t n = 1;; ++n) {
    if (hpc_mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    if (*abort) return false;
    if ((n & 7u) == 0u && hpc_globaltimer() - t0 > limit_ns) {
      hpc_status_set(status, HPC_ERR_TIMEOUT);
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void hpc_fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// generic-proxy shared-memory writes -> visible to the async proxy (TMA, MMA)
__device__ __forceinline__ void hpc_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- TMA ------------------------------------------------------------------
// 2-D tiled load; c0 is the inner (element) coordinate and must be a
// multiple of 16 bytes / element size.
__device__ __forceinline__ void hpc_tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                                int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(hpc_smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(hpc_smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void hpc_prefetch_tensormap(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- tensor memory ----------------------------------------------------------
// Whole warp.  Writes the allocated base address into *dst (shared memory).
__device__ __forceinline__ void hpc_tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   hpc_smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void hpc_tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void hpc_tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void hpc_tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- MMA ------------------------------------------------------------------
// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1 (bits 46-47), swizzle mode in
// bits 61-63 (0 none, 2 = 128-byte, 4 = 64-byte, 6 = 32-byte).
__device__ __forceinline__ uint64_t hpc_umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                                  uint32_t swizzle) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(swizzle & 7u) << 61;
  return d;
}

// Instruction descriptor, dense MMA with FP32 accumulation: a_fmt / b_fmt
// (kind::f16: 0 = F16, 1 = BF16; kind::tf32: 2 = TF32), both operands
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t hpc_umma_idesc(uint32_t a_fmt, uint32_t b_fmt, int N, int M) {
  return (1u << 4) | (a_fmt << 7) | (b_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void hpc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D (+)= A . B with A and B both BF16 from shared memory (kind::f16; the
// instruction descriptor names the BF16 formats), FP32 accumulation.
__device__ __forceinline__ void hpc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Asks the L2 cache to fetch `bytes` (a multiple of 16) from global memory
// at `p` (16-byte aligned); completes on its own, nothing waits for it.
__device__ __forceinline__ void hpc_prefetch_l2_bulk(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)),
               "r"(bytes)
               : "memory");
}

// Copies `bytes` (a multiple of 16) from global memory at `src` to this CTA's
// shared memory at `dst` (both 16-byte aligned) as one bulk copy, whose
// bytes complete the transaction count of *bar.
__device__ __forceinline__ void hpc_bulk_load(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          hpc_smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(hpc_smem_u32(bar))
      : "memory");
}

// Arrives once on *bar when every MMA issued so far by this thread is done.
__device__ __forceinline__ void hpc_mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          hpc_smem_u32(bar))
      : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane (warp w reads
// lanes 32 (w % 4) .. 32 (w % 4) + 31).
__device__ __forceinline__ void hpc_tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit TMEM columns of this thread's lane (the same lane
// rule as hpc_tmem_ld32).
__device__ __forceinline__ void hpc_tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of (row, byte-in-row) inside a K-major tile region whose rows
// are `row_bytes` (64 or 128) long, with the matching 16-byte-chunk XOR
// swizzle (the pattern TMA and the tensor core use on 1024-byte-aligned
// regions: address bits [4, 4+b) ^= bits [7, 7+b), b = 2 for 64-byte and 3
// for 128-byte rows).
__host__ __device__ __forceinline__ uint32_t hpc_swz_offset(uint32_t row, uint32_t byte,
                                                            uint32_t row_bytes) {
  const uint32_t a = row * row_bytes + byte;
  const uint32_t mask = row_bytes == 128 ? 7u : 3u;
  return a ^ (((a >> 7) & mask) << 4);
}
