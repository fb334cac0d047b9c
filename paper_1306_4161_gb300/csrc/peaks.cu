// Peak microbenchmarks: issue loops of one instruction kind on every SM, timed
// with CUDA events, to measure the roofline denominators this GPU does not
// publish (binary64 FMA and MMA, int8 MMA, bf16 mma.sync and tcgen05.mma) and
// the device copy bandwidth.
#include "internal.h"
#include "ptx.cuh"
#include "tc05.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

__global__ void __launch_bounds__(256) peak_dfma_kernel(int64_t iters, double *sink) {
  double a[8];
  const double x = 1.0 + 1e-12 * threadIdx.x, y = 1e-14;
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1e-3 * (i + 1 + threadIdx.x);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], x, y);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 1234.5678) sink[0] = s;
}

__global__ void __launch_bounds__(256) peak_dmma_kernel(int64_t iters, double *sink) {
  double c[4][4];
  const double a0 = 1e-3 * threadIdx.x, a1 = 2e-3, b0 = 1.0 + 1e-9;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = 0.0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
          "{%0,%1,%2,%3};"
          : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
          : "d"(a0), "d"(a1), "d"(b0));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += c[i][j];
  if (s == 1234.5678) sink[0] = s;
}

__global__ void __launch_bounds__(256) peak_imma_kernel(int64_t iters, int *sink) {
  int c[4][4];
  const uint32_t a = 0x01010101u * (threadIdx.x & 3), b = 0x01020102u;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = 0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += c[i][j];
  if (s == 123456789) sink[0] = s;
}

__global__ void __launch_bounds__(256) peak_hmma_kernel(int64_t iters, float *sink) {
  float c[4][4];
  const uint32_t a = 0x3f803f80u, b = 0x3f803f80u;   // bf16 pairs (1, 1)
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += c[i][j];
  if (s == 1234.5f) sink[0] = s;
}

// tcgen05 rate: one CTA per SM (its shared memory is more than half an SM's,
// so no second CTA can share the SM and its tensor memory), one thread issuing
// bf16 MMAs of the product kernels' shapes back to back: 128 x 256 x 16 on one
// SM, or 256 x 256 x 16 spanning a CTA pair.  The operands are small integers
// in [-128, 127] (the slice digits' form, exact in bf16), not zeros, since the
// rate under the power limit depends on the data.  Commits go out every 64
// MMAs and the issuer waits only for the group before, so the tensor pipe never
// drains between groups.  A single issuing thread reaches the full rate (one
// MMA per 128 cycles for both shapes), so this is also the product kernels'
// issue structure.
constexpr int TC_SMEM = 120 * 1024 + 1024 + 256;   // > half of an SM's 228 KB
constexpr int TC_GROUP = 64;                       // MMAs per commit

template <bool PAIR>
__global__ void __launch_bounds__(128, 1) peak_tc05_kernel(int64_t iters, int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 48 * 1024);   // 2 barriers
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 2);
  const int warp = threadIdx.x >> 5;
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  // operands: A (16 KB, 128 rows of 64 bf16) and B (32 KB) of small integers
  for (int i = threadIdx.x; i < 48 * 1024 / 4; i += blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u + 12345u * (rank + 1);
    h ^= h >> 13;
    h *= 0x5bd1e995u;
    h ^= h >> 15;
    const float lo = (float)((int)(h & 0xffu) - 128), hi = (float)((int)((h >> 8) & 0xffu) - 128);
    reinterpret_cast<uint32_t *>(smem)[i] = (__float_as_uint(lo) >> 16) |
                                           (__float_as_uint(hi) & 0xffff0000u);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar[0]), 1);
    mbar_init(smem_u32(&bar[1]), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    if (PAIR) {
      tmem_alloc2(smem_u32(slot), 512);
      tmem_relinquish2();
    } else {
      tmem_alloc(smem_u32(slot), 512);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *slot;
  if (PAIR) cluster_sync();
  if (threadIdx.x == 0 && (rank & 1u) == 0) {
    const uint32_t a = smem_u32(smem), b = a + 16 * 1024;
    const uint32_t idesc = idesc_bf16_f32(PAIR ? 256 : 128, 256);
    uint64_t ad[4], bd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ad[k] = sdesc_k128(a + k * 32);
      bd[k] = sdesc_k128(b + k * 32);
    }
    uint32_t ph[2] = {0u, 0u};
    int64_t grp = 0;
    bool ok = true;
    for (int64_t it = 0; it < iters && ok; it += 4) {
      // four k-steps into accumulator 0 or 1 (alternating every four)
      const uint32_t acc = tbase + (uint32_t)((it >> 2) & 1) * 256u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (PAIR)
          mma2_bf16(acc, ad[k], bd[k], idesc, k ? 1u : 0u);
        else
          mma_bf16(acc, ad[k], bd[k], idesc, k ? 1u : 0u);
      }
      if ((it + 4) % TC_GROUP == 0 || it + 4 >= iters) {
        const uint32_t bb = smem_u32(&bar[grp & 1]);
        if (PAIR)
          mma2_commit_mc(bb, (uint16_t)1u);
        else
          mma_commit(bb);
        if (grp >= 1) {   // the group before this one
          const int pb = (int)((grp - 1) & 1);
          ok = mbar_wait(smem_u32(&bar[pb]), ph[pb]);
          ph[pb] ^= 1u;
        }
        ++grp;
      }
    }
    if (ok && grp >= 1) {
      const int pb = (int)((grp - 1) & 1);
      ok = mbar_wait(smem_u32(&bar[pb]), ph[pb]);
    }
    if (!ok) record_error(status, HSUMMA_ERR_TIMEOUT, kSiteAccFull);
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();   // the pair's MMAs are complete before either CTA frees
  if (warp == 0) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc2(tbase, 512);
    else
      tmem_dealloc(tbase, 512);
  }
  if (PAIR) cluster_sync();
}

__global__ void copy_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

int run_peak(int kind, int64_t work, double *rate) {
  const int sms = state().sm_count;
  void *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 64);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(sink)");
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  double work_units = 0;
  void *buf = nullptr;
  int64_t n16 = 0;
  auto launch = [&](int64_t iters) {
    switch (kind) {
      case HSUMMA_PEAK_DFMA:
        peak_dfma_kernel<<<sms * 8, 256>>>(iters, (double *)sink);
        work_units = 2.0 * 8 * iters * sms * 8 * 256;
        break;
      case HSUMMA_PEAK_DMMA:
        peak_dmma_kernel<<<sms * 8, 256>>>(iters, (double *)sink);
        work_units = 2.0 * 16 * 8 * 4 * 4 * iters * sms * 8 * 8;
        break;
      case HSUMMA_PEAK_IMMA:
        peak_imma_kernel<<<sms * 8, 256>>>(iters, (int *)sink);
        work_units = 2.0 * 16 * 8 * 32 * 4 * iters * sms * 8 * 8;
        break;
      case HSUMMA_PEAK_HMMA_BF16:
        peak_hmma_kernel<<<sms * 8, 256>>>(iters, (float *)sink);
        work_units = 2.0 * 16 * 8 * 16 * 4 * iters * sms * 8 * 8;
        break;
      case HSUMMA_PEAK_TC05_BF16: {
        const int64_t it4 = iters < 4 ? 4 : (iters & ~int64_t(3));   // whole k-blocks
        peak_tc05_kernel<false><<<sms, 128, TC_SMEM>>>(it4, state().d_status);
        work_units = 2.0 * 128 * 256 * 16 * (double)it4 * sms;
        break;
      }
      case HSUMMA_PEAK_TC05_BF16_PAIR: {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(sms & ~1), 1, 1);
        cfg.blockDim = dim3(128, 1, 1);
        cfg.dynamicSmemBytes = TC_SMEM;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const int64_t it4 = iters < 4 ? 4 : (iters & ~int64_t(3));
        cudaLaunchKernelEx(&cfg, peak_tc05_kernel<true>, it4, state().d_status);
        work_units = 2.0 * 256 * 256 * 16 * (double)it4 * (sms / 2);
        break;
      }
      case HSUMMA_PEAK_COPY:
        copy_kernel<<<sms * 16, 512>>>((const uint4 *)buf, (uint4 *)buf + n16, n16);
        work_units = 2.0 * 16 * n16;
        break;
    }
  };
  int st = HSUMMA_OK;
  if (kind < HSUMMA_PEAK_DFMA || kind > HSUMMA_PEAK_TC05_BF16_PAIR) {
    set_error("unknown peak kind %d", kind);
    st = HSUMMA_ERR_ARG;
  }
  if (st == HSUMMA_OK && kind == HSUMMA_PEAK_TC05_BF16) {
    e = cudaFuncSetAttribute(peak_tc05_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaFuncSetAttribute");
  }
  if (st == HSUMMA_OK && kind == HSUMMA_PEAK_TC05_BF16_PAIR) {
    e = cudaFuncSetAttribute(peak_tc05_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaFuncSetAttribute");
  }
  if (st == HSUMMA_OK && kind == HSUMMA_PEAK_COPY) {
    // `work` MiB per buffer
    n16 = work * (1 << 20) / 16;
    e = cudaMalloc(&buf, 2 * n16 * 16);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(copy buffers)");
    else cudaMemset(buf, 0, 2 * n16 * 16);
  }
  if (st == HSUMMA_OK) {
    const int64_t iters = kind == HSUMMA_PEAK_COPY ? 1 : work;
    launch(iters > 4 ? iters / 4 : 1);  // warm-up
    cudaEventRecord(t0);
    launch(iters);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "peak kernel");
    } else {
      float ms = 0;
      cudaEventElapsedTime(&ms, t0, t1);
      *rate = work_units / (ms * 1e-3);
    }
  }
  if (buf) cudaFree(buf);
  cudaFree(sink);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return st;
}

}  // namespace hs
