// Inline-PTX building blocks for sm_103a: shared-memory barriers (mbarrier),
// Tensor Memory Accelerator copies (cp.async.bulk.tensor, with cluster
// multicast and L2 prefetch), cluster queries and barriers, and bounded waits.
// Every wait here gives up after a time limit and reports it, so that no kernel
// of this library can spin forever.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace hs {

// A bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 4000000000ull;

// Device status word layout: [0] status code, [1] site, [2] block, [3] extra.
enum DeviceSite : int {
  kSiteFull = 1,        // consumer waiting for a stage to be filled
  kSiteEmpty = 2,       // producer waiting for a stage to be released
  kSiteAccFull = 3,     // epilogue waiting for an accumulator
  kSiteAccEmpty = 4,    // MMA issuer waiting for an accumulator to be drained
  kSiteNonFinite = 5,   // split path saw Inf or NaN
};

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Record the first error of a launch (code < 0) and where it happened.
__device__ __forceinline__ void record_error(int *status, int code, int site) {
  if (atomicCAS(status, 0, code) == 0) {
    status[1] = site;
    status[2] = (int)(blockIdx.x + blockIdx.y * gridDim.x);
  }
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Arrive on the barrier at the same shared-memory offset in cluster CTA `rank`
// (the own CTA included), with release semantics at cluster scope.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar, uint32_t rank) {
  asm volatile(
      "{\n\t.reg .b32 ra;\n\t"
      "mapa.shared::cluster.u32 ra, %0, %1;\n\t"
      "mbarrier.arrive.release.cluster.shared::cluster.b64 _, [ra];\n\t}" ::"r"(bar),
      "r"(rank)
      : "memory");
}

// Arrive on the barrier at the same offset in CTA `rank` of the cluster without
// release ordering: for hand-backs that publish no memory writes (the arriving
// thread only read tensor memory, and its loads have completed).
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t bar, uint32_t rank) {
  asm volatile(
      "{\n\t.reg .b32 ra;\n\t"
      "mapa.shared::cluster.u32 ra, %0, %1;\n\t"
      "mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [ra];\n\t}" ::"r"(bar),
      "r"(rank)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with this parity to complete; false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// ---- Tensor Memory Accelerator ----
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm))
               : "memory");
}

// 2-D tiled load into this CTA's shared memory; completion counted in bytes on
// the local barrier.  x is the innermost (contiguous) coordinate.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm,
                                            int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// The same copy delivered to every CTA of the cluster whose bit is set in
// `mask`, at the same shared-memory offsets (data and barrier).
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap *tm,
                                               int32_t x, int32_t y, uint32_t bar,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar), "h"(mask)
      : "memory");
}

// Bring a tile into L2 without writing shared memory.
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *tm, int32_t x,
                                                int32_t y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(x), "r"(y)
               : "memory");
}

// ---- clusters ----
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_ctaid_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctaid.x;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_ctaid_y() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctaid.y;" : "=r"(r));
  return r;
}

// Whole-cluster barrier; every thread of every CTA of the cluster must call it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

// 64-bit load from the shared memory of cluster CTA `rank` at the address that
// `addr` has in this CTA.
__device__ __forceinline__ unsigned long long ld_shared_cluster_u64(uint32_t addr,
                                                                  uint32_t rank) {
  unsigned long long v;
  asm volatile(
      "{\n\t.reg .b32 ra;\n\t"
      "mapa.shared::cluster.u32 ra, %1, %2;\n\t"
      "ld.shared::cluster.u64 %0, [ra];\n\t}"
      : "=l"(v)
      : "r"(addr), "r"(rank)
      : "memory");
  return v;
}

// Named barrier among `nthreads` threads (a multiple of 32).
__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ORs a predicate over its `nthreads` threads: every
// participant gets the same answer, so they can leave a loop together.
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}

// Sleep for about `ns` nanoseconds (bounded by the timer, not by a flag).
__device__ __forceinline__ void bounded_sleep(unsigned long long ns) {
  const unsigned long long t0 = globaltimer();
  while (globaltimer() - t0 < ns) __nanosleep(1000);
}

// Warpgroup register reallocation (all 128 threads of the warpgroup execute it).
template <int N>
__device__ __forceinline__ void regs_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void regs_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}

// Which virtual processor a CTA plays.  Clusters are launched in cluster-index
// order; consecutive clusters are walked down columns of `rows` cluster rows,
// so the clusters resident at one time cover a square-ish part of C and the
// panels they stream stay in L2.  Returns the processor row r and column c of
// this CTA (its position inside the cluster is unchanged).
__device__ __forceinline__ void raster_proc(int cm, int cn, int cy, int cx, int rows,
                                            int *r, int *c) {
  const int ncx = (int)gridDim.x / cn, ncy = (int)gridDim.y / cm;
  const int L = ((int)blockIdx.y / cm) * ncx + (int)blockIdx.x / cn;
  const int group = L / (rows * ncx);
  const int in_group = min(rows, ncy - group * rows);
  const int idx = L - group * rows * ncx;
  const int gy = group * rows + idx % in_group, gx = idx / in_group;
  *r = gy * cm + cy;
  *c = gx * cn + cx;
}

// Layouts of the virtual grid.  Sub-tile i (of T rows) of processor row r
// starts at row *org; the rows of it that the processor owns and the matrix
// has are [org, org + T) ∩ [*lo, *hi).
//  block-checkerboard (Algorithm 1): the processor's block [r Mt, (r+1) Mt)
//    swept in tiles of T: org = r Mt + i T, [lo, hi) = the block;
//  block-cyclic (the distribution Section VI leaves to future work, with the
//    sub-tile as the distribution block): tile row r + i P, so
//    org = (r + i P) T and [lo, hi) = the tile.
// Columns use the same rule with (c, Q, Nt, N).
__device__ __forceinline__ void tile_rows(bool cyc, int r, int i, int P, int64_t Mt, int T,
                                          int64_t M, int64_t *org, int64_t *lo, int64_t *hi) {
  if (cyc) {
    *org = ((int64_t)r + (int64_t)i * P) * T;
    *lo = *org;
    *hi = *org + T < M ? *org + T : M;
  } else {
    *lo = (int64_t)r * Mt;
    *org = *lo + (int64_t)i * T;
    *hi = *lo + Mt < M ? *lo + Mt : M;
  }
}

// Whether the CTAs of a cluster whose first processor row is r0 all skip
// sub-step i: in the block-cyclic layout, when the cluster's first tile row
// lies at or past the end of the matrix (every later row of it does too).  The
// test depends on the cluster only, so a cluster skips in lockstep.
__device__ __forceinline__ bool tile_skipped(bool cyc, int r0, int i, int P, int T, int64_t M) {
  return cyc && ((int64_t)r0 + (int64_t)i * P) * T >= M;
}

// Owner of outer block q (starting at k index kq) among n processors: the
// processor column of the A block (n = Q) or row of the B block (n = P).
// Block-checkerboard: the processor whose k range [x Kblk, (x+1) Kblk) holds
// kq (Algorithm 1's pivot); block-cyclic: q mod n.
__device__ __forceinline__ int outer_owner(bool cyc, int64_t q, int64_t kq, int64_t Kblk, int n) {
  if (cyc) return (int)(q % n);
  const int64_t x = kq / Kblk;
  return x < n - 1 ? (int)x : n - 1;
}

// Byte offset of 16-byte chunk `chunk` (0..7) of row `row` inside a 128-byte
// swizzled tile (CU_TENSOR_MAP_SWIZZLE_128B): chunk index XOR (row mod 8).
__device__ __forceinline__ uint32_t swz128(uint32_t row, uint32_t byte_in_row) {
  return row * 128u + ((((byte_in_row >> 4) ^ (row & 7u)) << 4) | (byte_in_row & 15u));
}

}  // namespace hs
