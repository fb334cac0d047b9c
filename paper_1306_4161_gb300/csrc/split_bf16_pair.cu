// Split-precision HSUMMA, step 3 with bf16 slices on CTA pairs: the same exact
// diagonal sums as split_bf16.cu, for groups of two vertically adjacent
// processors (in-group grid 2 x 1), with every MMA spanning the pair's two SMs
// (tcgen05 cta_group::2, 256 x 256 x 16), and for groups of 2 x 2 processors
// as clusters of two such pairs (the three-level hierarchy: owners stage outer
// panels in L2, the cluster multicasts A along each processor row, the pair
// shares B through its MMA).
//
// The two processors of a group need the same 256 B columns and different A
// rows.  Each CTA loads its own 128 rows of A and one half (128 columns) of the
// group's B panel; the pair MMA reads both halves from the two SMs, which is
// the in-group column broadcast of Section III done by the tensor cores
// instead of a copy.  Each SM therefore holds 32 KB per k-stage (48 KB in the
// single-CTA kernel) and the ring is 6 stages deep: about 1.6 times the work
// in flight per byte of shared memory, and a third less traffic from L2.
//
// Synchronisation (no forwarding step): the first CTA of the pair ("leader")
// expects the bytes of both CTAs on its own "full" barrier, and the second
// CTA's copies count their bytes on that barrier directly (cta_group::2 bulk
// tensor copies).  Two issuing threads of the leader take the k-stages of
// parity 0 and 1 into separate accumulators (tensor-memory columns 0..255 and
// 256..511 of both SMs), with the staggered chunk ends of split_bf16.cu; each
// stage's MMA completion releases the stage in both CTAs, and each chunk end
// hands the accumulator to the drain warps of both CTAs, which return it to
// the leader.  Every wait is bounded (4 s) and ends in an error status.
//
// 2 x 2 groups: the two CTAs of a processor row each load one half (64 rows)
// of the row's A tile and multicast it to both (cta_group::2 copies that count
// the bytes on each destination's pair leader); a stage is released in all
// four CTAs once both pairs' MMAs have read it (the commits of both leaders,
// multicast to the cluster).
//
// Roles (384 threads per CTA): warp 0 issues the copies, warps 1 and 2 issue
// the MMAs (leader only; warp 1 of each CTA owns its tensor memory), warp 3
// idles, warps 4..11 drain their CTA's 128 rows into exact int32 planes.
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
constexpr int NEPI = 8;                // draining warps per CTA
constexpr int NTHREADS = (4 + NEPI) * 32;
constexpr int SEGST = 127 * CH;        // stages per int32 segment
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t IDESC2 = idesc_bf16_f32(2 * TM, TN);

struct PairParams {
  int32_t *D;
  int64_t M, N, K, Kpad, Mt, Nt, Kq, Kp;
  int P, Q, nsub_m, nsub_n, Bo, S, nkb, nseg;
  int d_lo, d_hi;                // the diagonals (slice pairs s + t = d) of this launch
  unsigned long long *counters;
  int *status;
};

__device__ __forceinline__ int64_t span(int64_t lo, int64_t hi, int64_t a, int64_t b) {
  const int64_t x = a > lo ? a : lo, y = b < hi ? b : hi;
  return y > x ? y - x : 0;
}

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              volatile int *abort_flag) {
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
}

// the chunk schedule of split_bf16.cu: issuer 0 closes a chunk every 16 of its
// stages, issuer 1 after 8 and then every 16; both at the segment's last stage
__device__ __forceinline__ bool chunk_end(int local, int seg_len) {
  const int c = (local >> 1) + 1;
  if (local + 2 >= seg_len) return true;
  return (local & 1) ? ((c + 8) % CH == 0) : (c % CH == 0);
}

// group tile L -> processor row r and column c of the CTA that is member `ry`
// of pair `px` of the group's cluster (CN pairs side by side): tiles walked
// down columns of 8 group rows
template <int CN>
__device__ __forceinline__ void tile_proc(int L, int ncx, int ncy, int ry, int px, int *r,
                                          int *c) {
  const int rows = 8;
  const int group = L / (rows * ncx);
  const int in_group = min(rows, ncy - group * rows);
  const int idx = L - group * rows * ncx;
  *r = (group * rows + idx % in_group) * 2 + ry;
  *c = (idx / in_group) * CN + px;
}

// CN pairs per cluster; CYC: block-cyclic layout of the grid, else block-checkerboard
template <int CN, bool CYC>
__global__ void __launch_bounds__(NTHREADS, 1)
    bf16_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmApf,
                     const __grid_constant__ CUtensorMap tmBpf, const PairParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *full = bars, *empty = bars + STAGES;
  uint64_t *acc_full = bars + 2 * STAGES, *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // cluster rank = 2 px + ry: pair px (the group's column), member ry (its row)
  const int rank = (int)cluster_ctarank();
  const int ry = rank & 1, px = rank >> 1;
  const bool leader = ry == 0;
  const int lead = rank & ~1;                     // this pair's first CTA
  const uint16_t all_mask = (uint16_t)((1u << (2 * CN)) - 1u);
  const uint16_t pair_mask = (uint16_t)(3u << lead);
  const uint16_t row_mask = CN == 2 ? (uint16_t)((1u << ry) | (1u << (ry + 2))) : (uint16_t)1u;
  const int ncx = p.Q / CN, ncy = p.P / 2, ntiles = ncx * ncy;
  const int ncl = (int)gridDim.x / (2 * CN), cid = (int)blockIdx.x / (2 * CN);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), CN);
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

  const int nkb = p.nkb;
  constexpr bool cyc = CYC;
  const int64_t nout = (p.Kpad + p.Bo - 1) / p.Bo;

  if (warp == 0) {
    // ---------------- copies (both CTAs) ----------------
    if (lane == 0) {
      unsigned long long a_ld = 0, a_dl = 0, b_ld = 0, pf = 0, nops = 0;
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (int L = cid; L < ntiles && ok; L += ncl) {
        int r, c;
        tile_proc<CN>(L, ncx, ncy, ry, px, &r, &c);
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          if (tile_skipped(cyc, r - ry, mi, p.P, TM, p.M)) continue;
          int64_t m0, row_lo, row_hi;
          tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
          const int64_t am0 = m0 + (CN == 2 ? px * (TM / 2) : 0);   // this CTA's A rows
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            if (tile_skipped(cyc, c - px, ni, p.Q, TN, p.N)) continue;
            int64_t n0, col_lo, col_hi;
            tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &n0, &col_lo, &col_hi);
            const int64_t nh = n0 + ry * HN;
            for (int d = p.d_lo; d <= p.d_hi && ok; ++d) {
              for (int s = 1; s < d && ok; ++s) {
                const int t = d - s;
                int rem = 0;   // k0 mod B, kept without a 64-bit division per stage
                for (int kb = 0; kb < nkb; ++kb) {
                  const int64_t k0 = (int64_t)kb * BKS;
                  const bool outer = rem == 0;
                  for (rem += BKS; rem >= p.Bo;) rem -= p.Bo;
                  if (outer) {
                    // owners stage the next outer panel into L2, one outer block
                    // ahead without gaps (the rule of split_bf16.cu)
                    const int64_t o = k0 / p.Bo;
                    int ns = s + 1, nd = d;
                    if (ns >= nd) { ++nd; ns = 1; }
                    const bool first = (d == p.d_lo && s == 1 && o == 0);
                    for (int w = first ? 0 : 1; w <= 1; ++w) {
                      int64_t q = o + w;
                      int ps = s, pt = t;
                      if (q >= nout) {
                        if (nd > p.d_hi) break;
                        q = 0;
                        ps = ns;
                        pt = nd - ns;
                      }
                      const int64_t kq = q * p.Bo, kend = imin64(p.Kpad, kq + p.Bo);
                      if (c == outer_owner(cyc, q, kq, p.Kq, p.Q)) {
                        for (int64_t kk = kq; kk < kend; kk += BKS)
                          tma_prefetch_3d(&tmApf, (int32_t)kk, (int32_t)m0, ps - 1);
                        pf += 1;
                      }
                      if (r == outer_owner(cyc, q, kq, p.Kp, p.P)) {
                        for (int64_t kk = kq; kk < kend; kk += BKS)
                          tma_prefetch_3d(&tmBpf, (int32_t)kk, (int32_t)n0, pt - 1);
                        pf += 1;
                      }
                    }
                  }
                  if (!wait_or_abort(smem_u32(&empty[stage]), phase ^ 1u, &abort_flag)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  const uint32_t a_dst = smem_u32(smem + stage * STAGE_BYTES);
                  const uint32_t b_dst = a_dst + A_BYTES;
                  // the pair leader's barrier counts the stage's bytes of both CTAs
                  const uint32_t fb = cluster_addr(smem_u32(&full[stage]), (uint32_t)lead);
                  if (leader) mbar_arrive_expect_tx(smem_u32(&full[stage]), 2 * STAGE_BYTES);
                  if (CN == 2) {
                    // half of the row's A tile, to both CTAs of the processor row
                    tma_load_3d_pair_mc(a_dst + px * (A_BYTES / 2), &tmA, (int32_t)k0,
                                        (int32_t)am0, s - 1, fb, row_mask);
                  } else if (leader) {
                    tma_load_3d(a_dst, &tmA, (int32_t)k0, (int32_t)m0, s - 1, fb);
                  } else {
                    tma_load_3d_pair(a_dst, &tmA, (int32_t)k0, (int32_t)m0, s - 1, fb);
                  }
                  if (leader)
                    tma_load_3d(b_dst, &tmB, (int32_t)k0, (int32_t)nh, t - 1, fb);
                  else
                    tma_load_3d_pair(b_dst, &tmB, (int32_t)k0, (int32_t)nh, t - 1, fb);
                  const int64_t kc = span(0, p.K, k0, k0 + BKS);
                  const int64_t ca = span(row_lo, row_hi, am0, am0 + TM / CN) * kc;
                  a_ld += ca;
                  a_dl += ca * CN;
                  b_ld += span(col_lo, col_hi, nh, nh + HN) * kc;
                  nops += 2;
                  if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
              }
            }
          }
        }
      }
      // tail: every release of the last stages has landed before leaving
      for (int i = 0; i < STAGES && ok; ++i) {
        if (!wait_or_abort(smem_u32(&empty[stage]), phase ^ 1u, &abort_flag)) {
          if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
          abort_flag = 1;
          ok = false;
        }
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
      // A rows reach the CN CTAs of their processor row in the cluster; each
      // half of B reaches both CTAs' products
      atomicAdd(&p.counters[0], a_ld);
      atomicAdd(&p.counters[1], a_dl);
      atomicAdd(&p.counters[2], b_ld);
      atomicAdd(&p.counters[3], 2 * b_ld);
      atomicAdd(&p.counters[4], pf);
      atomicAdd(&p.counters[5], nops);
    }
  } else if ((warp == 1 || warp == 2) && leader) {
    // ---------------- pair MMAs: issuer `me` takes the stages of parity me ----------------
    if (lane == 0) {
      const int me = warp - 1;
      uint32_t gst = 0, nchunk = 0;
      bool in_chunk = false;
      const uint32_t dt = tmem_base + (uint32_t)(me * TN);
      bool ok = true;
      for (int L = cid; L < ntiles && ok; L += ncl) {
        int r, c;
        tile_proc<CN>(L, ncx, ncy, ry, px, &r, &c);
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          if (tile_skipped(cyc, r - ry, mi, p.P, TM, p.M)) continue;
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            if (tile_skipped(cyc, c - px, ni, p.Q, TN, p.N)) continue;
            for (int d = p.d_lo; d <= p.d_hi && ok; ++d) {
              const int nst = (d - 1) * nkb;
              for (int st = 0; st < nst; ++st, ++gst) {
                if ((st & 1) != me) continue;
                const int seg_lo = st - st % SEGST;
                const int seg_len = min(nst, seg_lo + SEGST) - seg_lo;
                const int local = st - seg_lo;
                bool first = false;
                if (!in_chunk) {
                  if (!wait_or_abort(smem_u32(&acc_empty[me]), (nchunk & 1u) ^ 1u, &abort_flag)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteAccEmpty);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  in_chunk = true;
                  first = true;
                }
                const uint32_t stage = gst % STAGES, phase = (gst / STAGES) & 1u;
                if (!wait_or_abort(smem_u32(&full[stage]), phase, &abort_flag)) {
                  if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteFull);
                  abort_flag = 1;
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(smem + stage * STAGE_BYTES);
                const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
                for (int k = 0; k < BKS / 16; ++k) {
                  mma2_bf16(dt, sdesc_k128(a_addr + k * 32), sdesc_k128(b_addr + k * 32), IDESC2,
                            (first && k == 0) ? 0u : 1u);
                }
                mma2_commit_mc(smem_u32(&empty[stage]), all_mask);
                if (chunk_end(local, seg_len)) {
                  mma2_commit_mc(smem_u32(&acc_full[me]), pair_mask);
                  ++nchunk;
                  in_chunk = false;
                }
              }
            }
          }
        }
      }
    }
  } else if (warp >= 4) {
    // ---------------- drain (both CTAs): this SM's 128 rows -> exact int32 planes ----------------
    const int q = warp & 3;                 // tensor-memory lane quarter of this warp
    const int h = (warp - 4) >> 2;          // column half of the 256-column tile
    uint32_t nchunk0 = 0, nchunk1 = 0;
    bool ok = true;
    for (int L = cid; L < ntiles && ok; L += ncl) {
      int r, c;
      tile_proc<CN>(L, ncx, ncy, ry, px, &r, &c);
      for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
        if (tile_skipped(cyc, r - ry, mi, p.P, TM, p.M)) continue;
        int64_t m0, row_lo, row_hi;
        tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
        const int64_t row = m0 + q * 32 + lane;
        for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
          if (tile_skipped(cyc, c - px, ni, p.Q, TN, p.N)) continue;
          int64_t t0, col_lo, col_hi;
          tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &t0, &col_lo, &col_hi);
          const int64_t n0 = t0 + h * 128;
          const int64_t nvalid = imin64(128, imax64(0, col_hi - n0));
          for (int d = p.d_lo; d <= p.d_hi && ok; ++d) {
            const int nst = (d - 1) * nkb;
            for (int seg = 0; seg * SEGST < nst && ok; ++seg) {
              const int seg_len = min(nst, (seg + 1) * SEGST) - seg * SEGST;
              int acc[128];
#pragma unroll
              for (int i = 0; i < 128; ++i) acc[i] = 0;
              for (int local = 0; local < seg_len; ++local) {
                if (!chunk_end(local, seg_len)) continue;
                const int who = local & 1;
                const uint32_t par = who ? (nchunk1 & 1u) : (nchunk0 & 1u);
                // warp-uniform decision before the warp-collective tcgen05.ld
                const bool got = wait_or_abort(smem_u32(&acc_full[who]), par, &abort_flag);
                if (!__all_sync(0xffffffffu, got)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t ta =
                    tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(who * TN) + h * 128;
                // two 16-column loads in flight per wait: four round trips
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                  uint32_t v[16], w[16];
                  tmem_ld16(ta + j * 16, v);
                  tmem_ld16(ta + j * 16 + 16, w);
                  tmem_ld_wait();
#pragma unroll
                  for (int i = 0; i < 16; ++i) {
                    acc[j * 16 + i] += __float2int_rn(__uint_as_float(v[i]));
                    acc[j * 16 + 16 + i] += __float2int_rn(__uint_as_float(w[i]));
                  }
                }
                tc_fence_before();
                __syncwarp();
                // hand the accumulator back to the leader: the loads have completed
                // and nothing was written, so no release ordering is needed
                if (lane == 0) {
                  if (leader)
                    mbar_arrive(smem_u32(&acc_empty[who]));
                  else
                    mbar_arrive_cluster_relaxed(smem_u32(&acc_empty[who]), (uint32_t)lead);
                }
                if (who) ++nchunk1; else ++nchunk0;
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
  if (abort_flag) bounded_sleep(2000000ull);   // in-flight copies and MMAs land
  // both CTAs of the pair are done with tensor memory before it is released
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
  if (g.cm != 2 || (g.cn != 1 && g.cn != 2) || g.P % 2 || g.Q % g.cn) {
    set_error("the CTA-pair kernel needs groups realised as 2 x 1 or 2 x 2 clusters");
    return HSUMMA_ERR_ARG;
  }
  const int CN = g.cn;
  const int64_t Kpad = ceil_div(g.K, 64) * 64;
  const auto BF16 = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap tA, tB, tApf, tBpf;
  if (!encode_tmap_3d(&tA, BF16, 2, As, Kpad, g.M, S, BKS, TM / CN,
                      CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tB, BF16, 2, Bs, Kpad, g.N, S, BKS, HN, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tApf, BF16, 2, As, Kpad, g.M, S, BKS, TM, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_3d(&tBpf, BF16, 2, Bs, Kpad, g.N, S, BKS, TN, CU_TENSOR_MAP_SWIZZLE_NONE))
    return HSUMMA_ERR_ARG;
  PairParams p{};
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
  p.nsub_m = (int)(g.cyc ? ceil_div(ceil_div(g.M, TM), g.P) : ceil_div(g.Mt, TM));
  p.nsub_n = (int)(g.cyc ? ceil_div(ceil_div(g.N, TN), g.Q) : ceil_div(g.Nt, TN));
  p.Bo = g.Bo;
  p.S = S;
  p.nkb = (int)(Kpad / BKS);
  p.nseg = split_planes(g.K, S, HSUMMA_BF16_SLICES);
  p.counters = state().d_counters;
  p.status = state().d_status;
  auto kern = CN == 2 ? (g.cyc ? bf16_pair_kernel<2, true> : bf16_pair_kernel<2, false>)
                      : (g.cyc ? bf16_pair_kernel<1, true> : bf16_pair_kernel<1, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair smem)");
  cudaLaunchConfig_t cfg = {};
  const int ntiles = (g.P / 2) * (g.Q / CN);
  cfg.gridDim = dim3((unsigned)(2 * CN * ntiles), 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)(2 * CN);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // Long products run one launch per diagonal.  The hardware starts a cluster
  // whenever one finishes, so over many rounds of tiles the clusters resident
  // together drift apart, and with tiles of all S (S+1) / 2 slice pairs the L2
  // stops serving the panels they share: at 16384^3, S = 5, one launch read
  // 2.4 x the DRAM bytes of its tile rounds, one launch per diagonal 1.08 x
  // (a single round reads exactly its bytes either way).  Each launch repeats a
  // tile's fixed costs (tensor memory, barriers, pipeline fill, last drain),
  // which short or few-round products cannot afford.  Measured (ms, one launch
  // against one per diagonal): 1024 tiles x 15 x 16384 k: one launch faster by
  // 1 %; 2048 and 2304 tiles: per diagonal by 0.5-1.5 %; 3072 tiles x 15 x 8192
  // k: one launch by 1.3 %; 4096 tiles x 15 x 16384 k: per diagonal by 2-4 %.
  // Rule: per diagonal from 24 rounds and 15 x 16384 k-columns of pairs a tile.
  const int resident = state().sm_count / (2 * CN);
  const bool per_diagonal = resident > 0 && ntiles >= 24 * resident &&
                            (int64_t)(S * (S + 1) / 2) * Kpad >= 15 * 16384;
  for (int d = 2; d <= S + 1;) {
    p.d_lo = d;
    p.d_hi = per_diagonal ? d : S + 1;
    e = cudaLaunchKernelEx(&cfg, kern, tA, tB, tApf, tBpf, p);
    if (e != cudaSuccess) return cuda_fail(e, "launch bf16 pair kernel");
    count_launch();
    d = p.d_hi + 1;
  }
  return HSUMMA_OK;
}

}  // namespace hs
