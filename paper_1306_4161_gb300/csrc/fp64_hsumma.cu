// Native binary64 HSUMMA kernel (Section III, Algorithm 1) for sm_103a.
//
// One thread block (CTA) is one virtual processor P_(x,y)(i,j) of the P x Q
// grid; it owns the C block of rows [r Mt, (r+1) Mt) and columns
// [c Nt, (c+1) Nt) and sweeps it in 128 x 128 sub-tiles.  For every sub-tile
// the k loop runs in outer steps of Bouter columns and inner steps of b:
//   * outer step: the owner of the outer A block (Algorithm 1's
//     Pivot_group_col) brings A[rows, kB:(k+1)B] into L2 with a TMA prefetch,
//     the owner of the outer B block (Pivot_group_row) brings B[kB:(k+1)B, cols];
//     every group then reads the panels from L2 (the between-group broadcast);
//   * inner step: 16-wide slices of the panels are copied into shared memory
//     by the Tensor Memory Accelerator.  When the group is a thread-block
//     cluster, each A slice is fetched once per cluster row and multicast to the
//     Q/J CTAs of the row (row_comm), each B slice once per cluster column and
//     multicast to the P/I CTAs of the column (col_comm);
//   * local update (Algorithm 1's DGemm): c += a b with the binary64 tensor-core
//     instruction mma.sync.m16n8k4.f64 into register accumulators.
// The outer/inner structure does not change the arithmetic: every C element is
// the k-ascending binary64 sum of its products, so integer inputs give exact
// results for any G, b and Bouter.
//
// Roles: warps 0..7 compute (2 x 4 warps, 64 x 32 each); thread 0 also
// issues every copy: after each stage's release it refills whatever ring slots
// every receiving CTA has released (without waiting), and it waits only when
// the stage about to be multiplied has not been issued yet.  Eight warps put two on each SM
// sub-partition, which leaves a thread up to 255 registers (a ninth, copy-only
// warp would cap them at 168 and poll the barriers beside two compute warps).
// A 4-stage ring of 32 KB stages; "full" barriers count the bytes of a stage,
// "empty" barriers collect one release from every CTA that the stage's
// copies deliver to (its cluster row and column).
#include "internal.h"
#include "ptx.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int TM = 128, TN = 128, BK = 16, STAGES = 4;
constexpr int A_STAGE = TM * BK * 8;          // 16 KB: 16 pieces of 8 rows x 128 B
constexpr int B_STAGE = BK * TN * 8;          // 16 KB: 8 n-boxes x 2 pieces
constexpr int NTHREADS = 256;
constexpr int SMEM_BYTES = STAGES * (A_STAGE + B_STAGE) + 2 * STAGES * 8 + 1024;
constexpr int PF_K = 32;                      // k extent of one prefetch box

struct Fp64Params {
  double *C;
  int64_t ldc, M, N, K, Mt, Nt, Kq, Kp;
  int P, Q, cm, cn, nsub_m, nsub_n, Bo;
  unsigned long long *counters;
  int *status;
};

__device__ __forceinline__ void dmma(double (&c)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

__device__ __forceinline__ int64_t clamp_count(int64_t lo, int64_t hi, int64_t a, int64_t b) {
  // |[a, b) ∩ [lo, hi)|
  int64_t x = a > lo ? a : lo, y = b < hi ? b : hi;
  return y > x ? y - x : 0;
}

// The copy cursor of thread 0: the next k-stage of the sub-tile sweep to load
// into the ring, the ring slot it goes to, and the panel-load counters.
struct CopyCursor {
  int tile;                 // linear sub-tile index mi * nsub_n + ni (nsub_m * nsub_n: done)
  int64_t kt;               // k-stage within the sub-tile
  int rem;                  // k0 mod B, kept without a 64-bit division per stage
  int64_t m0, row_lo, row_hi, n0, col_lo, col_hi;
  uint32_t stage, phase;
  unsigned long long a_ld, a_dl, b_ld, b_dl, pf, nops;
};

// CYC: block-cyclic layout of the grid, else block-checkerboard
template <bool CYC>
__global__ void __launch_bounds__(NTHREADS, 1)
    fp64_hsumma_kernel(const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ CUtensorMap tmApf,
                       const __grid_constant__ CUtensorMap tmBpf, const Fp64Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_STAGE;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * (A_STAGE + B_STAGE));
  uint64_t *empty = full + STAGES;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cx = (int)cluster_ctaid_x(), cy = (int)cluster_ctaid_y();
  const int cn = p.cn, cm = p.cm;
  int r, c;
  raster_proc(cm, cn, cy, cx, 8, &r, &c);
  const uint16_t row_mask = (uint16_t)(((1u << cn) - 1u) << (cy * cn));
  uint16_t col_mask = 0;
  for (int y = 0; y < cm; ++y) col_mask |= (uint16_t)(1u << (y * cn + cx));

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), (uint32_t)(cn + cm - 1));
    }
    fence_mbar_init();
  }
  if (threadIdx.x == 32) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  cluster_sync();

  const int r0 = r - cy, c0 = c - cx;           // the cluster's first processor row / column
  // the block of a processor in the block-checkerboard layout (the epilogue
  // reads these; formed once here they cost the k loop no registers)
  const int64_t blk_row_lo = (int64_t)r * p.Mt, blk_row_hi = imin64(p.M, blk_row_lo + p.Mt);
  const int64_t blk_col_lo = (int64_t)c * p.Nt, blk_col_hi = imin64(p.N, blk_col_lo + p.Nt);
  constexpr bool cyc = CYC;
  const int64_t nk = (p.K + BK - 1) / BK;
  const int64_t nout = p.K > 0 ? (p.K + p.Bo - 1) / p.Bo : 0;
  const int ntile = p.nsub_m * p.nsub_n;

  // ---------------- copies (thread 0) ----------------
  CopyCursor cc = {};
  // place the cursor on the first sub-tile at or after cc.tile that is not skipped
  auto seek = [&]() {
    for (; cc.tile < ntile; ++cc.tile) {
      const int mi = cc.tile / p.nsub_n, ni = cc.tile - mi * p.nsub_n;
      if (tile_skipped(cyc, r0, mi, p.P, TM, p.M) || tile_skipped(cyc, c0, ni, p.Q, TN, p.N))
        continue;
      tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &cc.m0, &cc.row_lo, &cc.row_hi);
      tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &cc.n0, &cc.col_lo, &cc.col_hi);
      break;
    }
    cc.kt = 0;
    cc.rem = 0;
  };
  // issue the cursor's k-stage into its ring slot once every CTA the copies
  // reach has released the slot, then advance.  1: issued; 0: the slot is not
  // free yet (block = false only); -1: the wait ran out
  auto issue = [&](bool block) -> int {
    const uint32_t eb = smem_u32(&empty[cc.stage]);
    if (block) {
      if (!mbar_wait_cluster(eb, cc.phase ^ 1u)) return -1;
    } else if (!mbar_try_wait_cluster(eb, cc.phase ^ 1u)) {
      return 0;
    }
    const int64_t k0 = cc.kt * BK;
    const bool outer = cc.rem == 0;
    for (cc.rem += BK; cc.rem >= p.Bo;) cc.rem -= p.Bo;
    if (outer) {
      // outer step o: stage outer panel o (first step) and o + 1 into L2; the
      // owner of an outer block is the processor whose own block of A
      // (columns) / B (rows) contains its first index (block-cyclic: the
      // processor column / row q mod Q / q mod P)
      const int64_t o = k0 / p.Bo;
      for (int64_t q = (o == 0 ? 0 : o + 1); q <= o + 1 && q < nout; ++q) {
        const int64_t kq = q * p.Bo;
        const int64_t kend = imin64(p.K, kq + p.Bo);
        if (c == outer_owner(cyc, q, kq, p.Kq, p.Q)) {
          for (int64_t kk = kq; kk < kend; kk += PF_K)
            tma_prefetch_2d(&tmApf, (int32_t)kk, (int32_t)cc.m0);
          cc.pf += 1;
        }
        if (r == outer_owner(cyc, q, kq, p.Kp, p.P)) {
          for (int64_t kk = kq; kk < kend; kk += PF_K)
            tma_prefetch_2d(&tmBpf, (int32_t)cc.n0, (int32_t)kk);
          cc.pf += 1;
        }
      }
    }
    const uint32_t fb = smem_u32(&full[cc.stage]);
    mbar_arrive_expect_tx(fb, A_STAGE + B_STAGE);
    const uint32_t a_dst = smem_u32(sA + cc.stage * A_STAGE);
    const uint32_t b_dst = smem_u32(sB + cc.stage * B_STAGE);
    const int64_t kc = clamp_count(0, p.K, k0, k0 + BK);
    // A: 16 pieces of 8 rows x 16 k; piece i issued by cluster column i % cn
    for (int i = cx; i < TM / 8; i += cn) {
      const int64_t rr = cc.m0 + i * 8;
      if (cn > 1)
        tma_load_2d_mc(a_dst + i * 1024, &tmA, (int32_t)k0, (int32_t)rr, fb, row_mask);
      else
        tma_load_2d(a_dst + i * 1024, &tmA, (int32_t)k0, (int32_t)rr, fb);
      const int64_t cnt = clamp_count(cc.row_lo, cc.row_hi, rr, rr + 8) * kc;
      cc.a_ld += cnt;
      cc.a_dl += cnt * cn;
      cc.nops += 1;
    }
    // B: 8 n-boxes x 2 pieces of 8 k x 16 n; piece j issued by cluster row j % cm
    for (int j = cy; j < 2 * (TN / 16); j += cm) {
      const int64_t nn = cc.n0 + (j >> 1) * 16, kk = k0 + (j & 1) * 8;
      const uint32_t dst = b_dst + (j >> 1) * 2048 + (j & 1) * 1024;
      if (cm > 1)
        tma_load_2d_mc(dst, &tmB, (int32_t)nn, (int32_t)kk, fb, col_mask);
      else
        tma_load_2d(dst, &tmB, (int32_t)nn, (int32_t)kk, fb);
      const int64_t cnt =
          clamp_count(cc.col_lo, cc.col_hi, nn, nn + 16) * clamp_count(0, p.K, kk, kk + 8);
      cc.b_ld += cnt;
      cc.b_dl += cnt * cm;
      cc.nops += 1;
    }
    if (++cc.stage == STAGES) { cc.stage = 0; cc.phase ^= 1u; }
    if (++cc.kt == nk) {
      ++cc.tile;
      seek();
    }
    return 1;
  };
  // thread 0: stages issued so far; issue until stage `upto` is issued
  // (blocking) or while slots are free, never more than the ring holds beyond
  // the stages multiplied so far (a slot's barrier is then at most one phase
  // ahead, so its parity test cannot alias)
  int64_t issued = 0;
  bool copy_bad = false;        // thread 0: a wait for a free slot ran out
  auto refill = [&](int64_t upto, int64_t cap, bool block) {
    while (!copy_bad && cc.tile < ntile && issued < cap && (!block || issued <= upto)) {
      const int rc = issue(block && issued <= upto);
      if (rc < 0) {
        copy_bad = true;
        record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
      }
      if (rc <= 0) break;
      ++issued;
    }
  };
  if (threadIdx.x == 0) {
    if (nk > 0) seek();
    else cc.tile = ntile;
    refill(STAGES - 1, STAGES, true);           // the first STAGES stages
  }

  // ---------------- rank-16 updates with DMMA (all warps) ----------------
  const int wm = warp >> 2, wn = warp & 3;     // 2 x 4 warps, 64 x 32 each
  const int g = lane >> 2, t = lane & 3;
  uint32_t stage = 0, phase = 0;
  int64_t gst = 0;              // stages multiplied so far
  bool ok = true;
  for (int mi = 0; mi < p.nsub_m; ++mi) {
    if (tile_skipped(cyc, r0, mi, p.P, TM, p.M)) continue;
    for (int ni = 0; ni < p.nsub_n; ++ni) {
      if (tile_skipped(cyc, c0, ni, p.Q, TN, p.N)) continue;
      double acc[4][4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.0;
      for (int64_t kt = 0; kt < nk; ++kt, ++gst) {
        // thread 0 makes sure this stage is issued; it does not wait for a
        // stage its copies could not issue
        if (threadIdx.x == 0) refill(gst, gst + STAGES, true);
        const bool bad = (threadIdx.x == 0 && copy_bad) || !mbar_wait(smem_u32(&full[stage]), phase);
        if (bad && !(threadIdx.x == 0 && copy_bad)) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteFull);
        // all threads decide together whether to go on
        if (named_barrier_or(2, NTHREADS, bad)) {
          ok = false;
          break;
        }
        const uint8_t *a_base = sA + stage * A_STAGE;
        const uint8_t *b_base = sB + stage * B_STAGE;
#pragma unroll
        for (int kk = 0; kk < BK / 4; ++kk) {
          const int k = kk * 4 + t;
          double af[4][2], bf[4];
#pragma unroll
          for (int mt = 0; mt < 4; ++mt) {
            const int row = wm * 64 + mt * 16 + g;
            af[mt][0] = *reinterpret_cast<const double *>(a_base + swz128(row, k * 8));
            af[mt][1] = *reinterpret_cast<const double *>(a_base + swz128(row + 8, k * 8));
          }
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int n = wn * 32 + nt * 8 + g;
            bf[nt] = *reinterpret_cast<const double *>(b_base + (n >> 4) * 2048 +
                                                       swz128(k, (n & 15) * 8));
          }
#pragma unroll
          for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) dmma(acc[mt][nt], af[mt][0], af[mt][1], bf[nt]);
        }
        // release the stage to every CTA that delivers into it, then refill
        // the slots that are free already
        named_barrier(1, NTHREADS);
        if (threadIdx.x == 0) {
          const uint32_t eb = smem_u32(&empty[stage]);
          for (int x = 0; x < cn; ++x) mbar_arrive_cluster(eb, (uint32_t)(cy * cn + x));
          for (int y = 0; y < cm; ++y)
            if (y != cy) mbar_arrive_cluster(eb, (uint32_t)(y * cn + cx));
          refill(gst + 1, gst + 1 + STAGES, false);
        }
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
      // epilogue: C := the sub-tile (beta = 0), rows/cols inside the block
      // (block-cyclic: inside the tile and the matrix)
      int64_t m0, row_lo, row_hi, n0, col_lo, col_hi;
      if (cyc) {
        tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
        tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &n0, &col_lo, &col_hi);
      } else {
        m0 = blk_row_lo + (int64_t)mi * TM, row_hi = blk_row_hi;
        n0 = blk_col_lo + (int64_t)ni * TN, col_hi = blk_col_hi;
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t row = m0 + wm * 64 + mt * 16 + g + h * 8;
          if (row >= row_hi) continue;
          double *crow = p.C + row * p.ldc;
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int64_t col = n0 + wn * 32 + nt * 8 + 2 * t;
            const double v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
            if (col + 1 < col_hi && ((reinterpret_cast<uintptr_t>(crow + col) & 15) == 0)) {
              *reinterpret_cast<double2 *>(crow + col) = make_double2(v0, v1);
            } else {
              if (col < col_hi) crow[col] = v0;
              if (col + 1 < col_hi) crow[col + 1] = v1;
            }
          }
        }
      }
    }
    if (!ok) break;
  }
  if (!ok) atomicExch(&abort_flag, 1);
  if (threadIdx.x == 0) {
    atomicAdd(&p.counters[0], cc.a_ld);
    atomicAdd(&p.counters[1], cc.a_dl);
    atomicAdd(&p.counters[2], cc.b_ld);
    atomicAdd(&p.counters[3], cc.b_dl);
    atomicAdd(&p.counters[4], cc.pf);
    atomicAdd(&p.counters[5], cc.nops);
  }
  __syncthreads();
  // an aborted CTA may still have copies in flight into its shared memory:
  // give them a bounded moment to land before leaving
  if (abort_flag) bounded_sleep(2000000ull);
  // no CTA leaves while a peer may still deliver into its shared memory or
  // arrive on its barriers
  cluster_sync();
}

}  // namespace

int fp64_cluster_limit(int *limit) {
  cudaError_t e = cudaFuncSetAttribute(fp64_hsumma_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  e = cudaFuncSetAttribute(fp64_hsumma_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(non-portable cluster)");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 16;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  e = cudaOccupancyMaxPotentialClusterSize(&n, fp64_hsumma_kernel<false>, &cfg);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxPotentialClusterSize");
  *limit = n;
  return HSUMMA_OK;
}

int launch_fp64_hsumma(const GridPlan &g, const double *A, int64_t lda, const double *B,
                       int64_t ldb, double *C, int64_t ldc, cudaStream_t s) {
  CUtensorMap tA, tB, tApf, tBpf;
  const auto F64 = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  if (!encode_tmap_2d(&tA, F64, 8, A, g.K, g.M, lda, 16, 8, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&tB, F64, 8, B, g.N, g.K, ldb, 16, 8, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&tApf, F64, 8, A, g.K, g.M, lda, PF_K, TM, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_2d(&tBpf, F64, 8, B, g.N, g.K, ldb, TN, PF_K, CU_TENSOR_MAP_SWIZZLE_NONE))
    return HSUMMA_ERR_ARG;
  Fp64Params p;
  p.C = C;
  p.ldc = ldc;
  p.M = g.M;
  p.N = g.N;
  p.K = g.K;
  p.Mt = g.Mt;
  p.Nt = g.Nt;
  p.Kq = g.Kq;
  p.Kp = g.Kp;
  p.P = g.P;
  p.Q = g.Q;
  p.cm = g.cm;
  p.cn = g.cn;
  p.nsub_m = (int)(g.cyc ? ceil_div(ceil_div(g.M, TM), g.P) : ceil_div(g.Mt, TM));
  p.nsub_n = (int)(g.cyc ? ceil_div(ceil_div(g.N, TN), g.Q) : ceil_div(g.Nt, TN));
  p.Bo = g.Bo;
  p.counters = state().d_counters;
  p.status = state().d_status;
  auto kern = g.cyc ? fp64_hsumma_kernel<true> : fp64_hsumma_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  if (g.cm * g.cn > 8) {
    e = cudaFuncSetAttribute(kern,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(non-portable cluster)");
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.Q, (unsigned)g.P, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)g.cn;
  at[0].val.clusterDim.y = (unsigned)g.cm;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, tA, tB, tApf, tBpf, p);
  if (e != cudaSuccess) return cuda_fail(e, "launch fp64_hsumma_kernel");
  count_launch();
  return HSUMMA_OK;
}

}  // namespace hs
