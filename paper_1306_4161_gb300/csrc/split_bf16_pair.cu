// Split-precision HSUMMA, step 3 with bf16 slices, CTA-pair variant: the same
// exact diagonal products as split_bf16.cu, with every MMA spanning two SMs
// (tcgen05 cta_group::2, 256 x 256 x 16).
//
// The group cluster is laid out with its x dimension along processor rows, so
// the hardware's CTA pairs (cluster ranks 2k, 2k+1) are two vertically adjacent
// processors of one group: they need the same B columns and different A rows.
// Each CTA of a pair loads its own 128 rows of A (multicast along its cluster
// row, the in-group row broadcast) and one half (128 columns) of the pair's
// 256-column B panel (multicast to the CTAs of its cluster column that hold
// the same half, the in-group column broadcast); the pair's MMA reads both
// halves of B from the two SMs, so each SM's shared memory holds 32 KB per
// k-stage instead of 48 KB and the pipeline is 6 stages deep.
//
// Synchronisation: every CTA's "full" barrier counts the bytes of its own
// stage; the second CTA of a pair forwards its completion to the first
// ("pair full"), whose single thread issues the pair MMAs; the MMA completion
// is committed to the "empty" barriers of every CTA of the cluster (a stage is
// refilled once every pair of the cluster has consumed it) and, per
// accumulator chunk, to both CTAs' "acc full" barriers.  Both CTAs drain their
// own tensor memory (128 rows x 256 columns) exactly as in split_bf16.cu and
// release the accumulator to the first CTA of the pair.
#include "internal.h"
#include "ptx.cuh"
#include "tc05.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int TM = 128, TN = 256, HN = TN / 2, BKS = 64, STAGES = 6;
constexpr int A_BYTES = TM * BKS * 2, BH_BYTES = HN * BKS * 2;
constexpr int STAGE_BYTES = A_BYTES + BH_BYTES;
constexpr int CH = 16;                 // k-stages per accumulator chunk (1024 products)
constexpr int NEPI = 8;
constexpr int NTHREADS = (2 + NEPI) * 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;
constexpr uint32_t IDESC2 = idesc_bf16_f32(2 * TM, TN);

struct PairParams {
  int32_t *D;
  int64_t M, N, K, Kpad, Mt, Nt, Kq, Kp;
  int P, Q, cm, cn, nsub_m, nsub_n, Bo, S, nkb, seg_chunks, nseg;
  unsigned long long *counters;
  int *status;
};

__device__ __forceinline__ int64_t span(int64_t lo, int64_t hi, int64_t a, int64_t b) {
  const int64_t x = a > lo ? a : lo, y = b < hi ? b : hi;
  return y > x ? y - x : 0;
}

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              volatile int *abort_flag, bool cluster_scope) {
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (cluster_scope ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))
      return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
}

// cluster tile L -> processor row r and column c of this CTA (tiles walked
// down columns of 8 cluster rows); ry, rx: the CTA's row and column in the
// group cluster
__device__ __forceinline__ void tile_proc(int L, int ncx, int ncy, int cm, int cn, int ry,
                                          int rx, int *r, int *c) {
  const int rows = 8;
  const int group = L / (rows * ncx);
  const int in_group = min(rows, ncy - group * rows);
  const int idx = L - group * rows * ncx;
  *r = (group * rows + idx % in_group) * cm + ry;
  *c = (idx / in_group) * cn + rx;
}

__global__ void __launch_bounds__(NTHREADS, 1)
    bf16_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmApf,
                     const __grid_constant__ CUtensorMap tmBpf, const PairParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *full = bars, *empty = bars + STAGES, *pfull = bars + 2 * STAGES;
  uint64_t *acc_full = bars + 3 * STAGES, *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cm = p.cm, cn = p.cn;
  // cluster x runs along processor rows: rank = ry + rx cm, pairs differ in ry's low bit
  const int ry = (int)cluster_ctaid_x(), rx = (int)cluster_ctaid_y();
  const int rank = ry + rx * cm;
  const bool leader = (ry & 1) == 0;
  const int lead_rank = rank & ~1;
  const int half = ry & 1;                 // which 128 columns of B this CTA holds
  const int hw = cm / 2;                   // CTAs of a cluster column holding one half
  const int hj = ry >> 1;                  // index among them
  uint16_t a_mask = 0, b_mask = 0;
  for (int x = 0; x < cn; ++x) a_mask |= (uint16_t)(1u << (ry + x * cm));
  for (int y = half; y < cm; y += 2) b_mask |= (uint16_t)(1u << (y + rx * cm));
  const uint16_t all_mask = (uint16_t)((1u << (cm * cn)) - 1u);
  const uint16_t pair_mask = (uint16_t)(3u << lead_rank);
  const int ncx = p.Q / cn, ncy = p.P / cm, ntiles = ncx * ncy;
  const int ncl = (int)gridDim.x / cm, cid = (int)blockIdx.x / cm;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), (uint32_t)(cm * cn / 2));
      mbar_init(smem_u32(&pfull[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 2 * NEPI);
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc2(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish2();
  }
  if (threadIdx.x == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  cluster_sync();

  const int S = p.S, nkb = p.nkb;
  const int64_t nout = (p.Kpad + p.Bo - 1) / p.Bo;
  const bool a_contig = (TM / 8) % cn == 0, b_contig = (HN / 8) % hw == 0;
  const int a_box = a_contig ? TM / cn : 8, b_box = b_contig ? HN / hw : 8;

  if (warp == 0) {
    // ---------------- copies ----------------
    if (lane == 0) {
      unsigned long long a_ld = 0, a_dl = 0, b_ld = 0, b_dl = 0, pf = 0, nops = 0;
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (int L = cid; L < ntiles && ok; L += ncl) {
        int r, c;
        tile_proc(L, ncx, ncy, cm, cn, ry, rx, &r, &c);
        const int64_t row_lo = (int64_t)r * p.Mt, row_hi = imin64(p.M, row_lo + p.Mt);
        const int64_t col_lo = (int64_t)c * p.Nt, col_hi = imin64(p.N, col_lo + p.Nt);
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          const int64_t m0 = row_lo + (int64_t)mi * TM;
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            const int64_t n0 = col_lo + (int64_t)ni * TN;
            const int64_t nh = n0 + half * HN;
            for (int d = 2; d <= S + 1 && ok; ++d) {
              for (int s = 1; s < d && ok; ++s) {
                const int t = d - s;
                for (int kb = 0; kb < nkb; ++kb) {
                  const int64_t k0 = (int64_t)kb * BKS;
                  if (k0 % p.Bo == 0) {
                    const int64_t o = k0 / p.Bo;
                    for (int64_t q = (o == 0 ? 0 : o + 1); q <= o + 1 && q < nout; ++q) {
                      const int64_t kq = q * p.Bo, kend = imin64(p.Kpad, kq + p.Bo);
                      if (c == (int)imin64(p.Q - 1, kq / p.Kq)) {
                        for (int64_t kk = kq; kk < kend; kk += BKS)
                          tma_prefetch_3d(&tmApf, (int32_t)kk, (int32_t)m0, s - 1);
                        pf += 1;
                      }
                      // one B panel per processor column: its first row owns it
                      if (r == (int)imin64(p.P - 1, kq / p.Kp)) {
                        for (int64_t kk = kq; kk < kend; kk += BKS)
                          tma_prefetch_3d(&tmBpf, (int32_t)kk, (int32_t)n0, t - 1);
                        pf += 1;
                      }
                    }
                  }
                  if (!wait_or_abort(smem_u32(&empty[stage]), phase ^ 1u, &abort_flag, true)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  const uint32_t fb = smem_u32(&full[stage]);
                  mbar_arrive_expect_tx(fb, STAGE_BYTES);
                  const uint32_t a_base = smem_u32(smem + stage * STAGE_BYTES);
                  const uint32_t b_base = a_base + A_BYTES;
                  const int64_t kc = span(0, p.K, k0, k0 + BKS);
                  for (int i = a_contig ? rx * (a_box / 8) : rx; i < TM / 8;
                       i += a_contig ? TM / 8 : cn) {
                    const int64_t ar = m0 + (int64_t)i * 8;
                    const uint32_t dst = a_base + i * 8 * 128;
                    if (cn > 1)
                      tma_load_3d_mc(dst, &tmA, (int32_t)k0, (int32_t)ar, s - 1, fb, a_mask);
                    else
                      tma_load_3d(dst, &tmA, (int32_t)k0, (int32_t)ar, s - 1, fb);
                    const int64_t ca = span(row_lo, row_hi, ar, ar + a_box) * kc;
                    a_ld += ca;
                    a_dl += ca * cn;
                    nops += 1;
                  }
                  for (int i = b_contig ? hj * (b_box / 8) : hj; i < HN / 8;
                       i += b_contig ? HN / 8 : hw) {
                    const int64_t br = nh + (int64_t)i * 8;
                    const uint32_t dst = b_base + i * 8 * 128;
                    if (hw > 1)
                      tma_load_3d_mc(dst, &tmB, (int32_t)k0, (int32_t)br, t - 1, fb, b_mask);
                    else
                      tma_load_3d(dst, &tmB, (int32_t)k0, (int32_t)br, t - 1, fb);
                    // every loaded half is read by both CTAs of each pair it reaches
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
      }
      for (int i = 0; i < STAGES && ok; ++i) {
        if (!wait_or_abort(smem_u32(&empty[stage]), phase ^ 1u, &abort_flag, true)) {
          if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
          abort_flag = 1;
          ok = false;
        }
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
      atomicAdd(&p.counters[0], a_ld);
      atomicAdd(&p.counters[1], a_dl);
      atomicAdd(&p.counters[2], b_ld);
      atomicAdd(&p.counters[3], b_dl);
      atomicAdd(&p.counters[4], pf);
      atomicAdd(&p.counters[5], nops);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, gc = 0;
      bool ok = true;
      for (int L = cid; L < ntiles && ok; L += ncl) {
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            for (int d = 2; d <= S + 1 && ok; ++d) {
              const int nst = (d - 1) * nkb;
              for (int st = 0; st < nst; ++st) {
                if (!leader) {
                  // ---- second CTA of the pair: forward "stage filled" to the first
                  if (!wait_or_abort(smem_u32(&full[stage]), phase, &abort_flag, false)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteFull);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  mbar_arrive_cluster(smem_u32(&pfull[stage]), (uint32_t)lead_rank);
                  if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                  continue;
                }
                // ---- first CTA of the pair: issue the pair MMAs
                const uint32_t buf = gc & 1u;
                if (st % CH == 0) {
                  if (!wait_or_abort(smem_u32(&acc_empty[buf]), ((gc >> 1) & 1u) ^ 1u,
                                     &abort_flag, true)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteAccEmpty);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                }
                if (!wait_or_abort(smem_u32(&full[stage]), phase, &abort_flag, false) ||
                    !wait_or_abort(smem_u32(&pfull[stage]), phase, &abort_flag, true)) {
                  if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteFull);
                  abort_flag = 1;
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(smem + stage * STAGE_BYTES);
                const uint32_t b_addr = a_addr + A_BYTES;
                const uint32_t dt = tmem_base + buf * TN;
#pragma unroll
                for (int k = 0; k < BKS / 16; ++k) {
                  mma2_bf16(dt, sdesc_k128(a_addr + k * 32), sdesc_k128(b_addr + k * 32), IDESC2,
                            (st % CH != 0 || k > 0) ? 1u : 0u);
                }
                mma2_commit_mc(smem_u32(&empty[stage]), all_mask);
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                if (st % CH == CH - 1 || st == nst - 1) {
                  mma2_commit_mc(smem_u32(&acc_full[buf]), pair_mask);
                  ++gc;
                }
              }
            }
          }
        }
      }
    }
  } else {
    // ---------------- drain: tensor memory -> exact int32 planes ----------------
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    uint32_t gc = 0;
    bool ok = true;
    for (int L = cid; L < ntiles && ok; L += ncl) {
      int r, c;
      tile_proc(L, ncx, ncy, cm, cn, ry, rx, &r, &c);
      const int64_t row_lo = (int64_t)r * p.Mt, row_hi = imin64(p.M, row_lo + p.Mt);
      const int64_t col_lo = (int64_t)c * p.Nt, col_hi = imin64(p.N, col_lo + p.Nt);
      for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
        const int64_t row = row_lo + (int64_t)mi * TM + q * 32 + lane;
        for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
          const int64_t n0 = col_lo + (int64_t)ni * TN + h * 128;
          const int64_t nvalid = imin64(128, imax64(0, col_hi - n0));
          for (int d = 2; d <= S + 1 && ok; ++d) {
            const int nch = ((d - 1) * nkb + CH - 1) / CH;
            for (int seg = 0; seg * p.seg_chunks < nch && ok; ++seg) {
              const int c1 = min(nch, (seg + 1) * p.seg_chunks);
              int acc[128];
#pragma unroll
              for (int i = 0; i < 128; ++i) acc[i] = 0;
              for (int ch = seg * p.seg_chunks; ch < c1; ++ch) {
                const uint32_t buf = gc & 1u;
                const bool got =
                    wait_or_abort(smem_u32(&acc_full[buf]), (gc >> 1) & 1u, &abort_flag, true);
                if (!__all_sync(0xffffffffu, got)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + buf * TN + h * 128;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  uint32_t v[16];
                  tmem_ld16(ta + j * 16, v);
                  tmem_ld_wait();
#pragma unroll
                  for (int i = 0; i < 16; ++i)
                    acc[j * 16 + i] += __float2int_rn(__uint_as_float(v[i]));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(smem_u32(&acc_empty[buf]), (uint32_t)lead_rank);
                ++gc;
              }
              if (!ok) break;
              if (row < row_hi) {
                int32_t *drow =
                    p.D + ((int64_t)((d - 2) * p.nseg + seg) * p.M + row) * p.N + n0;
                if (nvalid == 128 && (reinterpret_cast<uintptr_t>(drow) & 15) == 0) {
#pragma unroll
                  for (int i = 0; i < 128; i += 4)
                    *reinterpret_cast<int4 *>(drow + i) =
                        make_int4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
                } else {
#pragma unroll
                  for (int i = 0; i < 128; ++i)
                    if (i < nvalid) drow[i] = acc[i];
                }
              }
            }
          }
        }
      }
    }
    if (!ok) {
      if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteAccFull);
      abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag) bounded_sleep(2000000ull);
  // both CTAs of every pair are done with tensor memory before it is released
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc2(tmem_base, TMEM_COLS);
  }
  cluster_sync();
}

}  // namespace

int launch_split_bf16_pair(const GridPlan &g, int S, const void *As, const void *Bs, int32_t *D,
                           cudaStream_t s) {
  const int64_t Kpad = ceil_div(g.K, 64) * 64;
  const int hw = g.cm / 2;
  const int a_box = (TM / 8) % g.cn == 0 ? TM / g.cn : 8;
  const int b_box = (HN / 8) % hw == 0 ? HN / hw : 8;
  const auto BF16 = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap tA, tB, tApf, tBpf;
  if (!encode_tmap_3d(&tA, BF16, 2, As, Kpad, g.M, S, BKS, a_box, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tB, BF16, 2, Bs, Kpad, g.N, S, BKS, b_box, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tApf, BF16, 2, As, Kpad, g.M, S, BKS, TM, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_3d(&tBpf, BF16, 2, Bs, Kpad, g.N, S, BKS, TN, CU_TENSOR_MAP_SWIZZLE_NONE))
    return HSUMMA_ERR_ARG;
  PairParams p;
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
  p.nsub_m = (int)ceil_div(g.Mt, TM);
  p.nsub_n = (int)ceil_div(g.Nt, TN);
  p.Bo = g.Bo;
  p.S = S;
  p.nkb = (int)(Kpad / BKS);
  p.seg_chunks = kSegChunks;
  p.nseg = split_planes(g.K, S);
  p.counters = state().d_counters;
  p.status = state().d_status;
  cudaError_t e = cudaFuncSetAttribute(bf16_pair_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  if (g.cm * g.cn > 8) {
    e = cudaFuncSetAttribute(bf16_pair_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(non-portable cluster)");
  }
  // one cluster per cluster tile; cluster x along processor rows
  cudaLaunchConfig_t cfg = {};
  const int ntiles = (g.Q / g.cn) * (g.P / g.cm);
  cfg.gridDim = dim3((unsigned)(ntiles * g.cm), (unsigned)g.cn, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)g.cm;
  at[0].val.clusterDim.y = (unsigned)g.cn;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, bf16_pair_kernel, tA, tB, tApf, tBpf, p);
  if (e != cudaSuccess) return cuda_fail(e, "launch bf16_pair_kernel");
  return HSUMMA_OK;
}

}  // namespace hs
