// Split-precision HSUMMA, step 3 with int8 slices on the warp-level integer
// tensor-core instruction mma.sync.m16n8k32.s8.s8.s32 (tcgen05 has no int8
// kind on sm_103a).
//
// Same HSUMMA data movement as the other kernels: one CTA per virtual
// processor sweeping 128 x 128 sub-tiles; 128-wide k-stages of the slices
// (128 bytes per row, 128-byte swizzle) copied by the Tensor Memory
// Accelerator, multicast inside the group cluster, outer panels staged into L2
// by their owners.  Digits are integers of magnitude <= 64, products <= 2^12,
// so int32 register accumulators are exact for 2^18 products: a diagonal is cut
// into segments of 2048 stages (2^18 products) and every segment's sums are
// stored as one int32 plane D[d-2][seg][i][j].
//
// Roles: warps 0..7 compute (2 x 4 warps of 64 x 32, fragments by ldmatrix),
// warp 8 issues the copies.  4 stages of 32 KB.
#include "internal.h"
#include "ptx.cuh"
#include "tc05.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int TM = 128, TN = 128, BKS = 128, STAGES = 4;
constexpr int A_BYTES = TM * BKS, B_BYTES = TN * BKS;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NCONS = 256;
constexpr int NTHREADS = NCONS + 32;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2 * STAGES * 8 + 1024;
constexpr int SEG_STAGES = (1 << 18) / BKS;   // 2^18 products per int32 segment

struct Int8Params {
  int32_t *D;
  int64_t M, N, K, Kpad, Mt, Nt, Kq, Kp;
  int P, Q, cm, cn, nsub_m, nsub_n, Bo, S, nkb, nseg;
  unsigned long long *counters;
  int *status;
};

__device__ __forceinline__ int64_t span(int64_t lo, int64_t hi, int64_t a, int64_t b) {
  const int64_t x = a > lo ? a : lo, y = b < hi ? b : hi;
  return y > x ? y - x : 0;
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void imma(int (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                     uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// CYC: block-cyclic layout of the grid, else block-checkerboard
template <bool CYC>
__global__ void __launch_bounds__(NTHREADS, 1)
    int8_diag_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmApf,
                     const __grid_constant__ CUtensorMap tmBpf, const Int8Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
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
  if (threadIdx.x == NCONS) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  cluster_sync();

  const int r0 = r - cy, c0 = c - cx;           // the cluster's first processor row / column
  constexpr bool cyc = CYC;
  const int S = p.S, nkb = p.nkb;
  const int64_t nout = (p.Kpad + p.Bo - 1) / p.Bo;
  const bool a_contig = (TM / 8) % cn == 0, b_contig = (TN / 8) % cm == 0;
  const int a_box = a_contig ? TM / cn : 8, b_box = b_contig ? TN / cm : 8;

  if (warp == NCONS / 32) {
    // ---------------- copies ----------------
    if (lane == 0) {
      unsigned long long a_ld = 0, a_dl = 0, b_ld = 0, b_dl = 0, pf = 0, nops = 0;
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
        if (tile_skipped(cyc, r0, mi, p.P, TM, p.M)) continue;
        int64_t m0, row_lo, row_hi;
        tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
        for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
          if (tile_skipped(cyc, c0, ni, p.Q, TN, p.N)) continue;
          int64_t n0, col_lo, col_hi;
          tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &n0, &col_lo, &col_hi);
          for (int d = 2; d <= S + 1 && ok; ++d) {
            for (int s = 1; s < d && ok; ++s) {
              const int t = d - s;
              int rem = 0;   // k0 mod B, kept without a 64-bit division per stage
              for (int kb = 0; kb < nkb; ++kb) {
                const int64_t k0 = (int64_t)kb * BKS;
                const bool outer = rem == 0;
                for (rem += BKS; rem >= p.Bo;) rem -= p.Bo;
                if (outer) {
                  const int64_t o = k0 / p.Bo;
                  for (int64_t q = (o == 0 ? 0 : o + 1); q <= o + 1 && q < nout; ++q) {
                    const int64_t kq = q * p.Bo, kend = imin64(p.Kpad, kq + p.Bo);
                    if (c == outer_owner(cyc, q, kq, p.Kq, p.Q)) {
                      for (int64_t kk = kq; kk < kend; kk += BKS)
                        tma_prefetch_3d(&tmApf, (int32_t)kk, (int32_t)m0, s - 1);
                      pf += 1;
                    }
                    if (r == outer_owner(cyc, q, kq, p.Kp, p.P)) {
                      for (int64_t kk = kq; kk < kend; kk += BKS)
                        tma_prefetch_3d(&tmBpf, (int32_t)kk, (int32_t)n0, t - 1);
                      pf += 1;
                    }
                  }
                }
                if (!mbar_wait_cluster(smem_u32(&empty[stage]), phase ^ 1u)) {
                  record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
                  ok = false;
                  break;
                }
                const uint32_t fb = smem_u32(&full[stage]);
                mbar_arrive_expect_tx(fb, STAGE_BYTES);
                const uint32_t a_base = smem_u32(smem + stage * STAGE_BYTES);
                const uint32_t b_base = a_base + A_BYTES;
                const int64_t kc = span(0, p.K, k0, k0 + BKS);
                for (int i = a_contig ? cx * (a_box / 8) : cx; i < TM / 8;
                     i += a_contig ? TM / 8 : cn) {
                  const int64_t ar = m0 + (int64_t)i * 8;
                  if (cn > 1)
                    tma_load_3d_mc(a_base + i * 1024, &tmA, (int32_t)k0, (int32_t)ar, s - 1, fb,
                                   row_mask);
                  else
                    tma_load_3d(a_base + i * 1024, &tmA, (int32_t)k0, (int32_t)ar, s - 1, fb);
                  const int64_t ca = span(row_lo, row_hi, ar, ar + a_box) * kc;
                  a_ld += ca;
                  a_dl += ca * cn;
                  nops += 1;
                }
                for (int i = b_contig ? cy * (b_box / 8) : cy; i < TN / 8;
                     i += b_contig ? TN / 8 : cm) {
                  const int64_t br = n0 + (int64_t)i * 8;
                  if (cm > 1)
                    tma_load_3d_mc(b_base + i * 1024, &tmB, (int32_t)k0, (int32_t)br, t - 1, fb,
                                   col_mask);
                  else
                    tma_load_3d(b_base + i * 1024, &tmB, (int32_t)k0, (int32_t)br, t - 1, fb);
                  const int64_t cb = span(col_lo, col_hi, br, br + b_box) * kc;
                  b_ld += cb;
                  b_dl += cb * cm;
                  nops += 1;
                }
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
              }
            }
          }
        }
      }
      if (!ok) atomicExch(&abort_flag, 1);
      atomicAdd(&p.counters[0], a_ld);
      atomicAdd(&p.counters[1], a_dl);
      atomicAdd(&p.counters[2], b_ld);
      atomicAdd(&p.counters[3], b_dl);
      atomicAdd(&p.counters[4], pf);
      atomicAdd(&p.counters[5], nops);
    }
  } else {
    // ---------------- consumers: int8 MMA, exact int32 sums ----------------
    const int wm = warp >> 2, wn = warp & 3;   // 2 x 4 warps, 64 x 32 each
    const int g = lane >> 2, t4 = lane & 3;
    // ldmatrix row addresses: lanes 0-7 / 8-15 / 16-23 / 24-31 feed matrices 0..3
    const int lrow = lane & 7, lmat = lane >> 3;
    uint32_t stage = 0, phase = 0;
    bool ok = true;
    for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
      if (tile_skipped(cyc, r0, mi, p.P, TM, p.M)) continue;
      int64_t m0, row_lo, row_hi;
      tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
      for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
        if (tile_skipped(cyc, c0, ni, p.Q, TN, p.N)) continue;
        int64_t n0, col_lo, col_hi;
        tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &n0, &col_lo, &col_hi);
        for (int d = 2; d <= S + 1 && ok; ++d) {
          const int nst = (d - 1) * nkb;
          // every plane of the diagonal is written: those past its own
          // segments as zeros (the recombination adds every plane)
          for (int seg = 0; seg < p.nseg && ok; ++seg) {
            const int st1 = min(nst, (seg + 1) * SEG_STAGES);
            int acc[4][4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[a][b][e] = 0;
            for (int st = seg * SEG_STAGES; st < st1; ++st) {
              const bool bad = !mbar_wait(smem_u32(&full[stage]), phase);
              if (bad) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteFull);
              if (named_barrier_or(2, NCONS, bad)) {
                ok = false;
                break;
              }
              const uint32_t a_base = smem_u32(smem + stage * STAGE_BYTES);
              const uint32_t b_base = a_base + A_BYTES;
#pragma unroll
              for (int kk = 0; kk < BKS / 32; ++kk) {
                uint32_t af[4][4], bfr[2][4];
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                  // matrices: rows +0/+8 (lmat & 1), k bytes +0/+16 (lmat >> 1)
                  const int row = wm * 64 + mt * 16 + (lmat & 1) * 8 + lrow;
                  const int kb = kk * 32 + (lmat >> 1) * 16;
                  ldsm_x4(a_base + row * 128 + ((((kb >> 4) ^ (row & 7))) << 4), af[mt]);
                }
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                  // two n8 tiles: matrices (n tile, k half) = (lmat >> 1, lmat & 1)
                  const int row = wn * 32 + np * 16 + (lmat >> 1) * 8 + lrow;
                  const int kb = kk * 32 + (lmat & 1) * 16;
                  ldsm_x4(b_base + row * 128 + ((((kb >> 4) ^ (row & 7))) << 4), bfr[np]);
                }
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                  for (int nt = 0; nt < 4; ++nt)
                    imma(acc[mt][nt], af[mt], bfr[nt >> 1][(nt & 1) * 2],
                         bfr[nt >> 1][(nt & 1) * 2 + 1]);
              }
              named_barrier(1, NCONS);
              if (threadIdx.x == 0) {
                const uint32_t eb = smem_u32(&empty[stage]);
                for (int x = 0; x < cn; ++x) mbar_arrive_cluster(eb, (uint32_t)(cy * cn + x));
                for (int y = 0; y < cm; ++y)
                  if (y != cy) mbar_arrive_cluster(eb, (uint32_t)(y * cn + cx));
              }
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            int32_t *Dp = p.D + (int64_t)((d - 2) * p.nseg + seg) * p.M * p.N;
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + wm * 64 + mt * 16 + g + h * 8;
                if (row >= row_hi) continue;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                  const int64_t col = n0 + wn * 32 + nt * 8 + 2 * t4;
                  int32_t *dp = Dp + row * p.N + col;
                  if (col + 1 < col_hi && (reinterpret_cast<uintptr_t>(dp) & 7) == 0) {
                    *reinterpret_cast<int2 *>(dp) = make_int2(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]);
                  } else {
                    if (col < col_hi) dp[0] = acc[mt][nt][2 * h];
                    if (col + 1 < col_hi) dp[1] = acc[mt][nt][2 * h + 1];
                  }
                }
              }
            }
          }
        }
      }
    }
    if (!ok) atomicExch(&abort_flag, 1);
  }
  __syncthreads();
  if (abort_flag) bounded_sleep(2000000ull);
  cluster_sync();
}

}  // namespace

int int8_cluster_limit(int *limit) {
  cudaError_t e = cudaFuncSetAttribute(int8_diag_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  e = cudaFuncSetAttribute(int8_diag_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  e = cudaOccupancyMaxPotentialClusterSize(&n, int8_diag_kernel<false>, &cfg);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxPotentialClusterSize");
  *limit = n;
  return HSUMMA_OK;
}

int launch_split_int8(const GridPlan &g, int S, const void *As, const void *Bs, int32_t *D,
                      cudaStream_t s) {
  const int64_t Kpad = ceil_div(g.K, 64) * 64;
  const int a_box = (TM / 8) % g.cn == 0 ? TM / g.cn : 8;
  const int b_box = (TN / 8) % g.cm == 0 ? TN / g.cm : 8;
  const auto I8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUtensorMap tA, tB, tApf, tBpf;
  if (!encode_tmap_3d(&tA, I8, 1, As, Kpad, g.M, S, BKS, a_box, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tB, I8, 1, Bs, Kpad, g.N, S, BKS, b_box, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tApf, I8, 1, As, Kpad, g.M, S, BKS, TM, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_3d(&tBpf, I8, 1, Bs, Kpad, g.N, S, BKS, TN, CU_TENSOR_MAP_SWIZZLE_NONE))
    return HSUMMA_ERR_ARG;
  Int8Params p;
  p.D = D;
  p.M = g.M;
  p.N = g.N;
  p.K = g.K;
  p.Kpad = Kpad;
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
  p.S = S;
  p.nkb = (int)ceil_div(Kpad, BKS);
  p.nseg = split_planes(g.K, S, HSUMMA_INT8_SLICES);
  p.counters = state().d_counters;
  p.status = state().d_status;
  auto kern = g.cyc ? int8_diag_kernel<true> : int8_diag_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  if (g.cm * g.cn > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1);
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
  if (e != cudaSuccess) return cuda_fail(e, "launch int8_diag_kernel");
  count_launch();
  return HSUMMA_OK;
}

}  // namespace hs
