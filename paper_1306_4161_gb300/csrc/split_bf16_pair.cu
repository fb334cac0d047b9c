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
// instead of a copy.  Each SM therefore needs 32 KB per 64 k-columns (48 KB in
// the single-CTA kernel), a third less traffic from L2 per product.
//
// A stage is two 64-column panels (128 k-columns, 64 KB per SM) and the ring
// holds 3: each operand of a stage arrives in one 32 KB copy through a 4-D
// "k-panel" tensor map that lands both panels one after the other.  An SM's
// copy engine takes about as long for a 16 KB copy as for a 32 KB one, so
// copies of single panels would cap the operand stream near 36 B per cycle,
// against the 64 B per cycle and SM that the full tensor rate needs here.
//
// Synchronisation (no forwarding step): the first CTA of the pair ("leader")
// expects the bytes of both CTAs on its own "full" barrier, and the second
// CTA's copies count their bytes on that barrier directly (cta_group::2 bulk
// tensor copies).  One issuing thread of the leader runs every MMA: a single
// thread sustains the full tensor rate (one 256 x 256 x 16 pair MMA per 128
// cycles), so the two accumulators (tensor-memory columns 0..255 and 256..511
// of both SMs) are used in turn, a chunk of at most 2 stages (256 products of
// digits of 9 bits) or 8 (1024 of 8 bits), the bound of exact fp32 sums, in
// each: while the drain warps of both CTAs
// empty one accumulator, the MMAs fill the other.  Each stage's MMA
// completion releases the stage in both CTAs, each chunk end hands the
// accumulator to the drain warps, and they return it to the leader.  Every
// wait is bounded (4 s) and ends in an error status.
//
// 2 x 2 groups: the two CTAs of a processor row each load one half (64 rows)
// of the row's A tile and multicast it to both (cta_group::2 copies that count
// the bytes on each destination's pair leader), one copy per panel, since a
// two-panel box of half a tile would not land in the MMA's layout; a stage is
// released in all four CTAs once both pairs' MMAs have read it (the commits of
// both leaders, multicast to the cluster).
//
// Roles (320 threads per CTA): warp 0 issues the copies, warp 1 issues the MMAs
// (leader only) and owns its CTA's tensor memory, warps 2..9 drain their CTA's
// 128 rows into exact int32 planes (a warp reads the tensor-memory lanes of
// its quarter, warp mod 4; warps 2..5 and 6..9 cover the 128 rows for the two
// column halves).  Ten warps leave 200 registers a thread, room for a drain
// warp's 128 sums and three 16-column loads in flight (12 warps with two idle
// ones, two loads in flight: 1-2 % slower with 9-bit digits).
//
// Work: a persistent launch runs one cluster per resident slot; each sweeps
// whole group tiles round robin with every diagonal of the launch, and a
// launch for all diagonals cuts the tiles of its last, part-filled round into
// one item per diagonal, dealt on the host to the least-loaded clusters (each
// item writes its own planes, so no sums meet across clusters).  All three
// roles walk the same item sequence.
#include <utility>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tc05.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int TM = 128, TN = 256, HN = TN / 2;
constexpr int PK = 64;                 // k-columns of a panel (128 bytes of bf16)
constexpr int KZ = 2;                  // panels per stage: one copy brings both
constexpr int BKS = PK * KZ;           // k-columns per stage
constexpr int STAGES = 3;
constexpr int A_PANEL = TM * PK * 2, B_PANEL = HN * PK * 2;   // 16 KB each
constexpr int A_BYTES = KZ * A_PANEL, BH_BYTES = KZ * B_PANEL;
constexpr int STAGE_BYTES = A_BYTES + BH_BYTES;
constexpr int NEPI = 8;                // draining warps per CTA
constexpr int NTHREADS = (2 + NEPI) * 32;   // copy warp, MMA warp, drain warps
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t IDESC2 = idesc_bf16_f32(2 * TM, TN);

// Tail schedule of a persistent launch: at most this many clusters and items.
constexpr int kMaxPairClusters = 160, kMaxTailItems = 640;

struct PairParams {
  int32_t *D;
  int64_t M, N, K, Kpad, Mt, Nt, Kq, Kp;
  int P, Q, nsub_m, nsub_n, Bo, S, nkb, nseg;
  int ch, segst;                 // stages per accumulator chunk (a power of two), per segment
  int d_lo, d_hi;                // the diagonals (slice pairs s + t = d) of this launch
  unsigned long long *counters;
  int *status;
  // work items: the tiles below `whole`, round robin over the clusters, each
  // with every diagonal of the launch; then cluster cid's tail items
  // [tail_off[cid], tail_off[cid + 1]), one tile and one diagonal each
  int whole;
  int16_t tail_off[kMaxPairClusters + 1];
  int32_t tail_L[kMaxTailItems];
  int8_t tail_d[kMaxTailItems];
};

// Work item i of cluster cid (of ncl): tile L and diagonals [dlo, dhi]; false
// past the cluster's last item.
__device__ __forceinline__ bool pair_item(const PairParams &p, int cid, int ncl, int i, int *L,
                                          int *dlo, int *dhi) {
  const int nw = p.whole > cid ? (p.whole - cid + ncl - 1) / ncl : 0;
  if (i < nw) {
    *L = cid + i * ncl;
    *dlo = p.d_lo;
    *dhi = p.d_hi;
    return true;
  }
  const int k = p.tail_off[cid] + (i - nw);
  if (k >= p.tail_off[cid + 1]) return false;
  *L = p.tail_L[k];
  *dlo = *dhi = p.tail_d[k];
  return true;
}

__device__ __forceinline__ int64_t span(int64_t lo, int64_t hi, int64_t a, int64_t b) {
  const int64_t x = a > lo ? a : lo, y = b < hi ? b : hi;
  return y > x ? y - x : 0;
}

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              volatile int *abort_flag) {
  // the first try needs no clock: most waits succeed at once
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
}

// a chunk closes after every `ch` stages of a segment and at its last stage;
// chunk n of the launch uses accumulator n mod 2
__device__ __forceinline__ bool chunk_end(int local, int seg_len, int ch) {
  return ((local + 1) & (ch - 1)) == 0 || local + 1 == seg_len;
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
                     const __grid_constant__ CUtensorMap tmBpf,
                     const __grid_constant__ PairParams p) {
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
  const int ncx = p.Q / CN, ncy = p.P / 2;
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
      int L, dlo, dhi;
      for (int it = 0; ok && pair_item(p, cid, ncl, it, &L, &dlo, &dhi); ++it) {
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
            // rows of A and columns of B this CTA copies for the sub-tile (inside
            // its block and the matrix); every slice pair delivers them over all K
            const int64_t a_rows = span(row_lo, row_hi, am0, am0 + TM / CN);
            const int64_t b_cols = span(col_lo, col_hi, nh, nh + HN);
            for (int d = dlo; d <= dhi && ok; ++d) {
              for (int s = 1; s < d && ok; ++s) {
                const int t = d - s;
                a_ld += (unsigned long long)(a_rows * p.K);
                a_dl += (unsigned long long)(a_rows * p.K * CN);
                b_ld += (unsigned long long)(b_cols * p.K);
                int rem = 0;   // panel start mod B, kept without a 64-bit division
                for (int kb = 0; kb < nkb; ++kb) {
                  const int64_t k0 = (int64_t)kb * BKS;
                  // outer steps fall on panel starts (B is a multiple of 64)
                  for (int h = 0; h < KZ; ++h) {
                    const int64_t kh = k0 + (int64_t)h * PK;
                    if (kh >= p.Kpad) break;
                    const bool outer = rem == 0;
                    for (rem += PK; rem >= p.Bo;) rem -= p.Bo;
                    if (!outer) continue;
                    // owners stage the next outer panel into L2, one outer block
                    // ahead without gaps (the rule of split_bf16.cu)
                    const int64_t o = kh / p.Bo;
                    int ns = s + 1, nd = d;
                    if (ns >= nd) { ++nd; ns = 1; }
                    const bool first = (d == dlo && s == 1 && o == 0);
                    for (int w = first ? 0 : 1; w <= 1; ++w) {
                      int64_t q = o + w;
                      int ps = s, pt = t;
                      if (q >= nout) {
                        if (nd > dhi) break;
                        q = 0;
                        ps = ns;
                        pt = nd - ns;
                      }
                      const int64_t kq = q * p.Bo, kend = imin64(p.Kpad, kq + p.Bo);
                      if (c == outer_owner(cyc, q, kq, p.Kq, p.Q)) {
                        for (int64_t kk = kq; kk < kend; kk += PK)
                          tma_prefetch_3d(&tmApf, (int32_t)kk, (int32_t)m0, ps - 1);
                        pf += 1;
                      }
                      if (r == outer_owner(cyc, q, kq, p.Kp, p.P)) {
                        for (int64_t kk = kq; kk < kend; kk += PK)
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
                  // (a panel past Kpad, at the end of an odd panel count, is
                  // zero-filled by the copy and counts in full)
                  const uint32_t fb = cluster_addr(smem_u32(&full[stage]), (uint32_t)lead);
                  if (leader) mbar_arrive_expect_tx(smem_u32(&full[stage]), 2 * STAGE_BYTES);
                  const int32_t kz0 = (int32_t)(k0 / PK);
                  if (CN == 2) {
                    // half (64 rows) of the row's A tile, panel by panel, to both
                    // CTAs of the processor row
                    for (int h = 0; h < KZ; ++h)
                      tma_load_4d_pair_mc(a_dst + h * A_PANEL + px * (A_PANEL / 2), &tmA, 0,
                                          (int32_t)am0, kz0 + h, s - 1, fb, row_mask);
                  } else if (leader) {
                    tma_load_4d(a_dst, &tmA, 0, (int32_t)m0, kz0, s - 1, fb);
                  } else {
                    tma_load_4d_pair(a_dst, &tmA, 0, (int32_t)m0, kz0, s - 1, fb);
                  }
                  if (leader)
                    tma_load_4d(b_dst, &tmB, 0, (int32_t)nh, kz0, t - 1, fb);
                  else
                    tma_load_4d_pair(b_dst, &tmB, 0, (int32_t)nh, kz0, t - 1, fb);
                  nops += CN == 2 ? KZ + 1 : 2;
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
  } else if (warp == 1 && leader) {
    // ---------------- pair MMAs: one issuer, the accumulators in turn ----------------
    if (lane == 0) {
      uint32_t gst = 0, nchunk = 0, dt = tmem_base;
      bool in_chunk = false;
      bool ok = true;
      // panels that lie inside Kpad in the last stage of a pair (2 unless the
      // panel count is odd)
      const int last_panels = (int)((p.Kpad - (int64_t)(nkb - 1) * BKS) / PK);
      int L, dlo, dhi;
      for (int it = 0; ok && pair_item(p, cid, ncl, it, &L, &dlo, &dhi); ++it) {
        int r, c;
        tile_proc<CN>(L, ncx, ncy, ry, px, &r, &c);
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          if (tile_skipped(cyc, r - ry, mi, p.P, TM, p.M)) continue;
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            if (tile_skipped(cyc, c - px, ni, p.Q, TN, p.N)) continue;
            for (int d = dlo; d <= dhi && ok; ++d) {
              const int nst = (d - 1) * nkb;
              int kb = 0;   // stage within the pair
              for (int st = 0; st < nst; ++st, ++gst) {
                const int npan = kb == nkb - 1 ? last_panels : KZ;
                if (++kb == nkb) kb = 0;
                const int seg_lo = st - st % p.segst;
                const int seg_len = min(nst, seg_lo + p.segst) - seg_lo;
                const int local = st - seg_lo;
                bool first = false;
                if (!in_chunk) {
                  // accumulator nchunk & 1, for the (nchunk >> 1)-th time
                  const uint32_t acc = nchunk & 1u;
                  if (!wait_or_abort(smem_u32(&acc_empty[acc]), ((nchunk >> 1) & 1u) ^ 1u,
                                     &abort_flag)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteAccEmpty);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  dt = tmem_base + acc * (uint32_t)TN;
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
                for (int h = 0; h < KZ; ++h) {
                  if (h >= npan) break;
#pragma unroll
                  for (int k = 0; k < PK / 16; ++k) {
                    mma2_bf16(dt, sdesc_k128(a_addr + h * A_PANEL + k * 32),
                              sdesc_k128(b_addr + h * B_PANEL + k * 32), IDESC2,
                              (first && h == 0 && k == 0) ? 0u : 1u);
                  }
                }
                mma2_commit_mc(smem_u32(&empty[stage]), all_mask);
                if (chunk_end(local, seg_len, p.ch)) {
                  mma2_commit_mc(smem_u32(&acc_full[nchunk & 1u]), pair_mask);
                  ++nchunk;
                  in_chunk = false;
                }
              }
            }
          }
        }
      }
    }
  } else if (warp >= 2) {
    // ---------------- drain (both CTAs): this SM's 128 rows -> exact int32 planes ----------------
    const int q = warp & 3;                 // tensor-memory lane quarter of this warp
    const int h = (warp - 2) >> 2;          // column half of the 256-column tile
    uint32_t nchunk = 0;
    bool ok = true;
    int L, dlo, dhi;
    for (int it = 0; ok && pair_item(p, cid, ncl, it, &L, &dlo, &dhi); ++it) {
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
          for (int d = dlo; d <= dhi && ok; ++d) {
            const int nst = (d - 1) * nkb;
            const int nseg_d = (nst + p.segst - 1) / p.segst;
            for (int seg = 0; seg < p.nseg && ok; ++seg) {
              const int seg_len =
                  seg < nseg_d ? min(nst, (seg + 1) * p.segst) - seg * p.segst : 0;
              uint32_t acc[128];
#pragma unroll
              for (int i = 0; i < 128; ++i) acc[i] = 0;
              // a plane past this diagonal's segments is written as zeros: the
              // recombination adds every plane of every diagonal
              for (int local = 0; local < seg_len; ++local) {
                if (!chunk_end(local, seg_len, p.ch)) continue;
                const uint32_t who = nchunk & 1u, par = (nchunk >> 1) & 1u;
                // warp-uniform decision before the warp-collective tcgen05.ld
                const bool got = wait_or_abort(smem_u32(&acc_full[who]), par, &abort_flag);
                if (!__all_sync(0xffffffffu, got)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t ta =
                    tmem_base + ((uint32_t)(q * 32) << 16) + who * (uint32_t)TN + h * 128;
                // three 16-column loads in flight per wait: three round trips
                float mx = 0.f;
#pragma unroll
                for (int j = 0; j < 8; j += 3) {
                  uint32_t v[3][16];
#pragma unroll
                  for (int r = 0; r < 3; ++r)
                    if (j + r < 8) tmem_ld16(ta + (j + r) * 16, v[r]);
                  tmem_ld_wait();
#pragma unroll
                  for (int r = 0; r < 3; ++r)
                    if (j + r < 8) drain_add16(acc + (j + r) * 16, v[r], mx);
                }
                if (__any_sync(0xffffffffu, !(mx < kFastDrainBound))) {
#pragma unroll
                  for (int j = 0; j < 8; j += 2) {
                    uint32_t v[16], w[16];
                    tmem_ld16(ta + j * 16, v);
                    tmem_ld16(ta + j * 16 + 16, w);
                    tmem_ld_wait();
                    drain_fix16(acc + j * 16, v);
                    drain_fix16(acc + j * 16 + 16, w);
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
                ++nchunk;
              }
              if (!ok) break;
              if (row < row_hi) {
                int32_t *drow =
                    p.D + ((int64_t)((d - 2) * p.nseg + seg) * p.M + row) * p.N + n0;
                if (nvalid == 128 && (reinterpret_cast<uintptr_t>(drow) & 15) == 0) {
#pragma unroll
                  for (int i = 0; i < 128; i += 4)
                    *reinterpret_cast<int4 *>(drow + i) =
                        make_int4((int)acc[i], (int)acc[i + 1], (int)acc[i + 2],
                                  (int)acc[i + 3]);
                } else {
#pragma unroll
                  for (int i = 0; i < 128; ++i)
                    if (i < nvalid) drow[i] = (int32_t)acc[i];
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

// Tail of a persistent one-launch product: the tiles past the last whole round
// (ntiles mod C of them, C resident clusters) would leave most clusters idle
// in a last part-filled round.  Instead each of those tiles is cut into one
// item per diagonal d (d - 1 slice pairs, its own planes, so no two clusters
// write the same sums), and the items go largest first to the cluster with
// the least work (every cluster starts with its whole tiles, S(S+1)/2 slice
// pairs each).  Fills p's tail items and returns true when that shortens the
// launch's longest cluster; leaves p as it is otherwise.
static bool tail_schedule(int ntiles, int C, int S, PairParams *p) {
  const int q = ntiles / C, rt = ntiles % C, W = S * (S + 1) / 2;
  if (rt == 0 || S < 2 || C > kMaxPairClusters || rt * S > kMaxTailItems) return false;
  std::vector<int> load(C, q * W);
  std::vector<std::vector<std::pair<int, int>>> items(C);
  for (int d = S + 1; d >= 2; --d)
    for (int t = 0; t < rt; ++t) {
      int best = 0;
      for (int c = 1; c < C; ++c)
        if (load[c] < load[best]) best = c;
      load[best] += d - 1;
      items[best].emplace_back(q * C + t, d);
    }
  int longest = 0;
  for (int c = 0; c < C; ++c) longest = load[c] > longest ? load[c] : longest;
  if (longest >= (q + 1) * W) return false;
  p->whole = q * C;
  int k = 0;
  for (int c = 0; c < C; ++c) {
    p->tail_off[c] = (int16_t)k;
    for (auto &it : items[c]) {
      p->tail_L[k] = it.first;
      p->tail_d[k] = (int8_t)it.second;
      ++k;
    }
  }
  p->tail_off[C] = (int16_t)k;
  return true;
}

// Clusters of the pair kernel (2 CN CTAs) that fit on the device at once,
// queried once per CN and kept.
int pair_resident_clusters(int CN, int *clusters) {
  int &res = state().pair_resident[CN == 2 ? 2 : 1];
  if (res == 0) {
    auto kern = CN == 2 ? bf16_pair_kernel<2, false> : bf16_pair_kernel<1, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair smem)");
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3((unsigned)(2 * CN), 1, 1);
    q.blockDim = dim3(NTHREADS, 1, 1);
    q.dynamicSmemBytes = SMEM_BYTES;
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = (unsigned)(2 * CN);
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &q);
    if (e != cudaSuccess || n < 1) {
      set_error("cudaOccupancyMaxActiveClusters(pair kernel): %s (%d clusters)",
                cudaGetErrorString(e), n);
      return HSUMMA_ERR_CUDA;
    }
    res = n;
  }
  *clusters = res;
  return HSUMMA_OK;
}

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
  // copies: KZ panels per copy (64 rows and one panel per copy for the A
  // halves of 2 x 2 groups); owner prefetches: one panel per instruction
  if (!encode_tmap_kpanels(&tA, BF16, 2, As, Kpad, g.M, S, TM / CN, CN == 2 ? 1 : KZ) ||
      !encode_tmap_kpanels(&tB, BF16, 2, Bs, Kpad, g.N, S, HN, KZ) ||
      !encode_tmap_3d(&tApf, BF16, 2, As, Kpad, g.M, S, PK, TM, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_3d(&tBpf, BF16, 2, Bs, Kpad, g.N, S, PK, TN, CU_TENSOR_MAP_SWIZZLE_NONE))
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
  p.nkb = (int)ceil_div(Kpad, BKS);
  p.nseg = split_planes(g.K, S, HSUMMA_BF16_SLICES);
  p.ch = bf16_chunk_products(slice_width(HSUMMA_BF16_SLICES, S)) / BKS;
  p.segst = kSegChunks * p.ch;
  p.counters = state().d_counters;
  p.status = state().d_status;
  auto kern = CN == 2 ? (g.cyc ? bf16_pair_kernel<2, true> : bf16_pair_kernel<2, false>)
                      : (g.cyc ? bf16_pair_kernel<1, true> : bf16_pair_kernel<1, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair smem)");
  cudaLaunchConfig_t cfg = {};
  const int ntiles = (g.P / 2) * (g.Q / CN);
  const int policy = state().pair_launch;
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
  // k: one launch by 1.3 %; 4096 tiles x 15 x 16384 k: per diagonal by 2-4 %;
  // 4096 tiles x 10 x 16384 k (S = 4): per diagonal by 2-5 %.
  // Rule: per diagonal from 24 rounds and 10 x 16384 k-columns of pairs a tile.
  const int resident = state().sm_count / (2 * CN);
  const int split = policy & 0xf;
  const bool per_diagonal =
      split == HSUMMA_PAIR_LAUNCH_PER_DIAGONAL ||
      (split == HSUMMA_PAIR_LAUNCH_AUTO && resident > 0 && ntiles >= 24 * resident &&
       (int64_t)(S * (S + 1) / 2) * Kpad >= 10 * 16384);
  p.whole = ntiles;
  int nclusters = ntiles;
  if (policy & HSUMMA_PAIR_PERSISTENT) {
    // one cluster per resident slot, each sweeping tiles L = cid, cid + ncl, ...
    int res = 0;
    const int st = pair_resident_clusters(CN, &res);
    if (st != HSUMMA_OK) return st;
    nclusters = ntiles < res ? ntiles : res;
    // one launch for all diagonals: the part-filled last round is spread
    // over every resident cluster
    if (!per_diagonal && tail_schedule(ntiles, res, S, &p)) nclusters = res;
  }
  cfg.gridDim = dim3((unsigned)(2 * CN * nclusters), 1, 1);
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
