// Inline-PTX wrappers for the 5th-generation tensor cores (tcgen05) of sm_103a:
// tensor-memory allocation, shared-memory matrix descriptors, the bf16 MMA with
// fp32 accumulation in tensor memory, commits to mbarriers and tensor-memory
// loads.
#pragma once

#include <cstdint>

namespace hs {

// Shared-memory matrix descriptor for a K-major tile written by the Tensor
// Memory Accelerator with 128-byte swizzling: rows of 128 bytes, groups of 8
// rows 1024 bytes apart (stride byte offset), descriptor version 1, layout
// "128B swizzle".  `saddr` is a shared-memory byte address; advancing along K
// inside the 128-byte row adds (bytes >> 4) to the start-address field.
__device__ __forceinline__ uint64_t sdesc_k128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)(16u >> 4) << 16;                 // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;               // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: bf16 A and B (both K-major), fp32 D,
// shape M x N (M = 128: one CTA, N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                        // D format: f32
         | (1u << 7)                      // A format: bf16
         | (1u << 10)                     // B format: bf16
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   dst_smem),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] x B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive (once) on a local mbarrier when every MMA issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// The same, arriving on the barrier at this offset in every CTA of `mask`.
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// 32 consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Drain of an accumulator chunk into this thread's exact 32-bit sums.  A
// value x of the chunk (an integer in fp32) with |x| < 2^22 converts by one
// floating-point add: x + 1.5 * 2^23 lies in (2^23, 2^24), where consecutive
// integers have consecutive encodings, so its bits are those of 1.5 * 2^23
// plus x.  drain_add16 adds 16 values that way and keeps the largest |x| in
// mx; when any lane of the warp saw one of 2^22 or more, the chunk is read
// again from tensor memory and drain_fix16 replaces every value's add by the
// float-to-int conversion instruction (which issues at a fraction of the add
// rate): the sums are exact either way, modulo 2^32 in between.
constexpr float kFastDrainBound = 4194304.f;   // 2^22
__device__ __forceinline__ uint32_t drain_fast_bits(float x) {
  return __float_as_uint(x + 12582912.f) - 0x4B400000u;   // 1.5 * 2^23 and its encoding
}
// Two values per step: one packed add (add.f32x2) converts both, one
// three-input max tracks them, against one add and one max per value (1-3 %
// faster products at 16384^3 with 9-bit digits, where a chunk is 2 stages).
__device__ __forceinline__ void drain_add16(uint32_t *acc, const uint32_t (&v)[16], float &mx) {
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    const float x0 = __uint_as_float(v[i]), x1 = __uint_as_float(v[i + 1]);
    asm("max.f32 %0, %1, %2, %3;" : "=f"(mx) : "f"(fabsf(x0)), "f"(fabsf(x1)), "f"(mx));
    unsigned long long y;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(y)
        : "l"(((unsigned long long)v[i + 1] << 32) | v[i]), "l"(0x4B4000004B400000ull));
    acc[i] += (uint32_t)y - 0x4B400000u;
    acc[i + 1] += (uint32_t)(y >> 32) - 0x4B400000u;
  }
}
__device__ __forceinline__ void drain_fix16(uint32_t *acc, const uint32_t (&v)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float x = __uint_as_float(v[i]);
    acc[i] += (uint32_t)__float2int_rn(x) - drain_fast_bits(x);
  }
}

// ---- CTA-pair (cta_group::2) forms: one MMA spans two SMs of a cluster (CTA
// ranks 2k and 2k+1); A is split along M (each CTA supplies 128 rows), B along
// N (each CTA supplies half of the columns), D rows land in each CTA's own
// tensor memory.  Allocation, relinquish and release are collective: one warp
// in each CTA of the pair executes them.
__device__ __forceinline__ void tmem_alloc2(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   dst_smem),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish2() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void mma2_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on the barrier at this offset in every CTA of `mask` once every
// pair MMA issued so far has completed.
__device__ __forceinline__ void mma2_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// 3-D tiled TMA load (x innermost), optionally multicast.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *tm, int32_t x,
                                            int32_t y, int32_t z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// shared::cluster address of the same shared-memory offset in CTA `rank` of
// the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t smem_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr), "r"(rank));
  return r;
}

// 3-D tile load into this CTA's shared memory whose bytes are counted on an
// mbarrier of the CTA pair (cta_group::2: `bar` is a shared::cluster address
// in this CTA or in its peer)
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const void *tm, int32_t x,
                                                 int32_t y, int32_t z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// 3-D tile load multicast to the CTAs in `mask`, whose bytes are counted, for
// each destination CTA, on the mbarrier at `bar`'s offset in the first CTA of
// that destination's CTA pair (cta_group::2)
__device__ __forceinline__ void tma_load_3d_pair_mc(uint32_t dst, const void *tm, int32_t x,
                                                    int32_t y, int32_t z, uint32_t bar,
                                                    uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster.cta_group::2 [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const void *tm, int32_t x,
                                               int32_t y, int32_t z, uint32_t bar,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(mask)
      : "memory");
}

// 4-D tiled loads over the k-panel view {64, rows, Kp / 64, S} of a slice
// tensor (see encode_tmap_kpanels): a box {64, rows, kz, 1} brings kz
// consecutive 64-column panels of a tile in one copy, landing as kz panels of
// rows x 128 bytes one after the other.  Plain, CTA-pair (bytes counted on the
// pair leader's barrier) and multicast CTA-pair forms, as for the 3-D loads.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *tm, int32_t x, int32_t y,
                                            int32_t z, int32_t w, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d_pair(uint32_t dst, const void *tm, int32_t x,
                                                 int32_t y, int32_t z, int32_t w, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d_pair_mc(uint32_t dst, const void *tm, int32_t x,
                                                    int32_t y, int32_t z, int32_t w,
                                                    uint32_t bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster.cta_group::2 [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_3d(const void *tm, int32_t x, int32_t y,
                                                int32_t z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

}  // namespace hs
