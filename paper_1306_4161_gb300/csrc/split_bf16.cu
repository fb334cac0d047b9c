// Split-precision HSUMMA, step 3 with bf16 slices on the tcgen05 tensor cores.
//
// For every C block the kernel forms the exact diagonal sums
//     D_d = sum_{s+t=d} A_s B_t,   d = 2 .. S+1,
// of the bf16 digit slices (integers of magnitude <= 2^(w-1): 256 for w = 9),
// with the same
// HSUMMA data movement as the binary64 kernel: one CTA per virtual processor
// (Section III), b-wide panels of each slice multicast inside the group
// cluster (inner level, Figure 4), outer panels staged into L2 by their owners
// (outer level, Figure 3).  The local update runs as tcgen05.mma
// (128 x 256 x 16, bf16 x bf16 -> fp32 in tensor memory).
//
// Exactness: a product of two digits is an integer of magnitude <= 2^(2w-2),
// so an fp32 accumulator that sums at most 2^(26-2w) of them per element (256
// for w = 9, 1024 for w = 8) stays an integer of magnitude <= 2^24 and is
// exact.  Accumulators are therefore drained into int32 registers after at
// most that many products ("chunk": 4 or 16 k-stages of 64); pairs of the
// same diagonal are concatenated along k.  A diagonal is cut into segments of
// 127 chunks (sums <= 127 * 2^24 < 2^31); each segment's exact int32 sums are
// stored as one plane of the output, D[d-2][seg][i][j], and the recombination
// adds the planes of a diagonal exactly.
//
// One MMA issuer.  A single issuing thread sustains the full tensor rate (one
// 128 x 256 x 16 MMA per 128 cycles), so the two accumulators (tensor-memory
// columns 0..255 and 256..511) are used in turn, chunk n in accumulator
// n mod 2: while the drain warps empty one, the MMAs fill the other.
//
// Roles (384 threads): warp 0 issues the copies, warp 1 issues the MMAs and
// owns tensor memory, warps 2 and 3 idle, warps 4..11 drain (a warp reads the
// tensor-memory lanes of its quarter, warp mod 4; warps 4..7 and 8..11 cover
// the 128 rows for the two column halves; 128 int32 sums per thread).  With
// 12 warps the compiler fits every role in 168 registers without spilling;
// with the idle warps left out it spills.
//
// Shared memory: a ring of 4 stages, the A slots (16 KB, 128 x 64) side by
// side and then the B slots (32 KB, 256 x 64).  What bounds this kernel is
// the delivery of its operands: 48 KB per 512-cycle stage (96 B per cycle at
// the full tensor rate, against about 70 that the copy engine of an SM
// streams, and about 360 cycles per copy), and the issuing thread's own path
// per stage.  Copies of two panels at once (measured) and two issuing threads
// (measured) were both slower for flat groups.
#include "internal.h"
#include "ptx.cuh"
#include "tc05.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int TM = 128, TN = 256, BKS = 64, STAGES = 4;
constexpr int A_BYTES = TM * BKS * 2, B_BYTES = TN * BKS * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int B_REGION = STAGES * A_BYTES;   // ring: all A slots, then all B slots
constexpr int NEPI = 8;                // draining warps
constexpr int NTHREADS = (4 + NEPI) * 32;   // copy warp, MMA warp, two idle warps, drain warps
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t IDESC = idesc_bf16_f32(TM, TN);

struct SplitParams {
  int32_t *D;
  int64_t M, N, K, Kpad, Mt, Nt, Kq, Kp;
  int P, Q, cm, cn, nsub_m, nsub_n, Bo, S, nkb, nseg;
  int ch, segst;   // k-stages per accumulator chunk (a power of two), per int32 segment
  unsigned long long *counters;
  int *status;
};

__device__ __forceinline__ int64_t span(int64_t lo, int64_t hi, int64_t a, int64_t b) {
  const int64_t x = a > lo ? a : lo, y = b < hi ? b : hi;
  return y > x ? y - x : 0;
}

// wait that also gives up as soon as another role of the CTA has aborted
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              volatile int *abort_flag, bool cluster_scope) {
  // the first try needs no clock: most waits succeed at once
  if (cluster_scope ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))
    return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (cluster_scope ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))
      return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
}

// Does stage `local` (counted from the start of its segment of `seg_len`
// stages) end a chunk?  A chunk closes after every `ch` stages of a segment
// and at its last stage.
__device__ __forceinline__ bool chunk_end(int local, int seg_len, int ch) {
  return ((local + 1) & (ch - 1)) == 0 || local + 1 == seg_len;
}

// cluster tile L -> processor row r and column c of this CTA: tiles are
// walked down columns of 8 cluster rows (see raster_proc)
__device__ __forceinline__ void tile_proc(int L, int ncx, int ncy, int cm, int cn, int cy,
                                          int cx, int *r, int *c) {
  const int rows = 8;
  const int group = L / (rows * ncx);
  const int in_group = min(rows, ncy - group * rows);
  const int idx = L - group * rows * ncx;
  *r = (group * rows + idx % in_group) * cm + cy;
  *c = (idx / in_group) * cn + cx;
}

// CYC: block-cyclic layout of the grid, else block-checkerboard; FLAT: groups
// served flat (no cluster), which folds the cluster arithmetic of the copy
// thread's per-stage path away
template <bool CYC, bool FLAT>
__global__ void __launch_bounds__(NTHREADS, 1)
    bf16_diag_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmApf,
                     const __grid_constant__ CUtensorMap tmBpf, const SplitParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *full = bars, *empty = bars + STAGES;
  uint64_t *acc_full = bars + 2 * STAGES, *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cx = (int)cluster_ctaid_x(), cy = (int)cluster_ctaid_y();
  const int cn = FLAT ? 1 : p.cn, cm = FLAT ? 1 : p.cm;
  // persistent clusters: cluster `cid` plays the virtual processors of the
  // cluster tiles L = cid, cid + ncl, ... (walked in raster order), so the
  // clusters resident together work on neighbouring blocks in step
  const int ncl = (int)gridDim.x / cn, cid = (int)blockIdx.x / cn;
  const int ncx = p.Q / cn, ncy = p.P / cm, ntiles = ncx * ncy;
  const uint16_t row_mask = (uint16_t)(((1u << cn) - 1u) << (cy * cn));
  uint16_t col_mask = 0;
  for (int y = 0; y < cm; ++y) col_mask |= (uint16_t)(1u << (y * cn + cx));
  const bool clustered = cn * cm > 1;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), (uint32_t)(cn + cm - 1));
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), NEPI);
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  if (threadIdx.x == 32 * 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  cluster_sync();

  const int S = p.S, nkb = p.nkb;
  constexpr bool cyc = CYC;
  const int64_t nout = (p.Kpad + p.Bo - 1) / p.Bo;
  // rows per TMA box: the CTA's contiguous share of a tile when the cluster
  // width divides the tile's 8-row pieces, else single 8-row pieces
  const bool a_contig = (TM / 8) % cn == 0, b_contig = (TN / 8) % cm == 0;
  const int a_box = a_contig ? TM / cn : 8, b_box = b_contig ? TN / cm : 8;

  if (warp == 0) {
    // ---------------- copies ----------------
    // One issuing thread at one stage per 512 cycles: everything that does not
    // change along k (the counted rows, the pieces of a clustered operand) is
    // worked out once per sub-tile, so that the per-stage path stays short.
    if (lane == 0) {
      unsigned long long a_ld = 0, a_dl = 0, b_ld = 0, b_dl = 0, pf = 0, nops = 0;
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (int L = cid; L < ntiles && ok; L += ncl) {
        int r, c;
        tile_proc(L, ncx, ncy, cm, cn, cy, cx, &r, &c);
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          if (tile_skipped(cyc, r - cy, mi, p.P, TM, p.M)) continue;
          int64_t m0, row_lo, row_hi;
          tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            if (tile_skipped(cyc, c - cx, ni, p.Q, TN, p.N)) continue;
            int64_t n0, col_lo, col_hi;
            tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &n0, &col_lo, &col_hi);
            // rows of A and columns of B this CTA copies for the sub-tile (its
            // share of the cluster row / column: a contiguous box, or 8-row
            // pieces dealt round robin), inside its block and the matrix; every
            // slice pair delivers them over all K
            int64_t a_rows = 0, b_cols = 0;
            for (int i = a_contig ? cx * (a_box / 8) : cx; i < TM / 8; i += a_contig ? TM / 8 : cn)
              a_rows += span(row_lo, row_hi, m0 + (int64_t)i * 8, m0 + (int64_t)i * 8 + a_box);
            for (int i = b_contig ? cy * (b_box / 8) : cy; i < TN / 8; i += b_contig ? TN / 8 : cm)
              b_cols += span(col_lo, col_hi, n0 + (int64_t)i * 8, n0 + (int64_t)i * 8 + b_box);
            for (int d = 2; d <= S + 1 && ok; ++d) {
              for (int s = 1; s < d && ok; ++s) {
                const int t = d - s;
                a_ld += (unsigned long long)(a_rows * p.K);
                a_dl += (unsigned long long)(a_rows * p.K * cn);
                b_ld += (unsigned long long)(b_cols * p.K);
                b_dl += (unsigned long long)(b_cols * p.K * cm);
                int rem = 0;   // k0 mod B, kept without a 64-bit division per stage
                for (int kb = 0; kb < nkb; ++kb) {
                  const int64_t k0 = (int64_t)kb * BKS;
                  const bool outer = rem == 0;
                  for (rem += BKS; rem >= p.Bo;) rem -= p.Bo;
                  if (outer) {
                    // outer step o of pair (s, t): the owners stage the next outer
                    // panel into L2 -- panel o + 1 of this pair, or, at the last
                    // outer step, panel 0 of the next pair of the sub-tile -- so the
                    // prefetch runs one outer block ahead without gaps; the sub-tile's
                    // very first panel is staged at its own start
                    const int64_t o = k0 / p.Bo;
                    int ns = s + 1, nd = d;            // next pair in the sweep order
                    if (ns >= nd) { ++nd; ns = 1; }
                    const bool first = (d == 2 && s == 1 && o == 0);
                    for (int w = first ? 0 : 1; w <= 1; ++w) {
                      int64_t q = o + w;
                      int ps = s, pt = t;
                      if (q >= nout) {
                        if (nd > S + 1) break;
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
                  if (!wait_or_abort(smem_u32(&empty[stage]), phase ^ 1u, &abort_flag, true)) {
                    if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteEmpty);
                    abort_flag = 1;
                    ok = false;
                    break;
                  }
                  const uint32_t fb = smem_u32(&full[stage]);
                  mbar_arrive_expect_tx(fb, STAGE_BYTES);
                  const uint32_t a_base = smem_u32(smem + stage * A_BYTES);
                  const uint32_t b_base = smem_u32(smem + B_REGION + stage * B_BYTES);
                  // A tile (128 rows): contiguous share of the cluster row, or 8-row
                  // pieces dealt round-robin when the width does not divide 16
                  for (int i = a_contig ? cx * (a_box / 8) : cx; i < TM / 8;
                       i += a_contig ? TM / 8 : cn) {
                    const uint32_t dst = a_base + i * 8 * 128;
                    const int32_t y = (int32_t)(m0 + (int64_t)i * 8);
                    if (cn > 1)
                      tma_load_3d_mc(dst, &tmA, (int32_t)k0, y, s - 1, fb, row_mask);
                    else
                      tma_load_3d(dst, &tmA, (int32_t)k0, y, s - 1, fb);
                    nops += 1;
                  }
                  for (int i = b_contig ? cy * (b_box / 8) : cy; i < TN / 8;
                       i += b_contig ? TN / 8 : cm) {
                    const uint32_t dst = b_base + i * 8 * 128;
                    const int32_t y = (int32_t)(n0 + (int64_t)i * 8);
                    if (cm > 1)
                      tma_load_3d_mc(dst, &tmB, (int32_t)k0, y, t - 1, fb, col_mask);
                    else
                      tma_load_3d(dst, &tmB, (int32_t)k0, y, t - 1, fb);
                    nops += 1;
                  }
                  if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
              }
            }
          }
        }
      }
      // tail: every release of the last stages has landed before leaving
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
    // ---------------- MMA issue: one thread, the accumulators in turn ----------------
    if (lane == 0) {
      uint32_t gst = 0;   // stage counter over the whole launch: ring slot and phase
      uint32_t nchunk = 0, dt = tmem_base;
      bool in_chunk = false;
      const uint16_t rel_mask = row_mask | col_mask;
      bool ok = true;
      for (int L = cid; L < ntiles && ok; L += ncl) {
        int r, c;
        tile_proc(L, ncx, ncy, cm, cn, cy, cx, &r, &c);
        for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
          if (tile_skipped(cyc, r - cy, mi, p.P, TM, p.M)) continue;
          for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
            if (tile_skipped(cyc, c - cx, ni, p.Q, TN, p.N)) continue;
            for (int d = 2; d <= S + 1 && ok; ++d) {
              const int nst = (d - 1) * nkb;
              for (int st = 0; st < nst; ++st, ++gst) {
                const int seg_lo = st - st % p.segst;
                const int seg_len = min(nst, seg_lo + p.segst) - seg_lo;
                const int local = st - seg_lo;
                bool first = false;
                if (!in_chunk) {
                  const uint32_t acc = nchunk & 1u;
                  if (!wait_or_abort(smem_u32(&acc_empty[acc]), ((nchunk >> 1) & 1u) ^ 1u,
                                     &abort_flag, false)) {
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
                if (!wait_or_abort(smem_u32(&full[stage]), phase, &abort_flag, false)) {
                  if (!abort_flag) record_error(p.status, HSUMMA_ERR_TIMEOUT, kSiteFull);
                  abort_flag = 1;
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(smem + stage * A_BYTES);
                const uint32_t b_addr = smem_u32(smem + B_REGION + stage * B_BYTES);
#pragma unroll
                for (int k = 0; k < BKS / 16; ++k) {
                  mma_bf16(dt, sdesc_k128(a_addr + k * 32), sdesc_k128(b_addr + k * 32), IDESC,
                           (first && k == 0) ? 0u : 1u);
                }
                // release the stage to every CTA that delivers into it
                if (clustered)
                  mma_commit_mc(smem_u32(&empty[stage]), rel_mask);
                else
                  mma_commit(smem_u32(&empty[stage]));
                if (chunk_end(local, seg_len, p.ch)) {
                  mma_commit(smem_u32(&acc_full[nchunk & 1u]));
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
    // ---------------- drain: chunk ends in stage order -> exact int32 planes ----------------
    const int q = warp & 3;                 // tensor-memory lane quarter of this warp
    const int h = (warp - 4) >> 2;          // column half
    uint32_t nchunk = 0;
    bool ok = true;
    for (int L = cid; L < ntiles && ok; L += ncl) {
      int r, c;
      tile_proc(L, ncx, ncy, cm, cn, cy, cx, &r, &c);
      for (int mi = 0; mi < p.nsub_m && ok; ++mi) {
        if (tile_skipped(cyc, r - cy, mi, p.P, TM, p.M)) continue;
        int64_t m0, row_lo, row_hi;
        tile_rows(cyc, r, mi, p.P, p.Mt, TM, p.M, &m0, &row_lo, &row_hi);
        const int64_t row = m0 + q * 32 + lane;
        for (int ni = 0; ni < p.nsub_n && ok; ++ni) {
          if (tile_skipped(cyc, c - cx, ni, p.Q, TN, p.N)) continue;
          int64_t t0, col_lo, col_hi;
          tile_rows(cyc, c, ni, p.Q, p.Nt, TN, p.N, &t0, &col_lo, &col_hi);
          const int64_t n0 = t0 + h * 128;
          const int64_t nvalid = imin64(128, imax64(0, col_hi - n0));
          for (int d = 2; d <= S + 1 && ok; ++d) {
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
                // the whole warp decides together: tcgen05.ld below is warp-collective
                const bool got = wait_or_abort(smem_u32(&acc_full[who]), par, &abort_flag, false);
                if (!__all_sync(0xffffffffu, got)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t ta =
                    tmem_base + ((uint32_t)(q * 32) << 16) + who * (uint32_t)TN + h * 128;
                // two 16-column loads in flight per wait: four round trips
                float mx = 0.f;
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                  uint32_t v[16], w[16];
                  tmem_ld16(ta + j * 16, v);
                  tmem_ld16(ta + j * 16 + 16, w);
                  tmem_ld_wait();
                  drain_add16(acc + j * 16, v, mx);
                  drain_add16(acc + j * 16 + 16, w, mx);
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
                if (lane == 0) mbar_arrive(smem_u32(&acc_empty[who]));
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
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
  cluster_sync();
}

}  // namespace

int bf16_cluster_limit(int *limit) {
  cudaError_t e = cudaFuncSetAttribute(bf16_diag_kernel<false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  e = cudaFuncSetAttribute(bf16_diag_kernel<false, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  e = cudaOccupancyMaxPotentialClusterSize(&n, bf16_diag_kernel<false, false>, &cfg);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxPotentialClusterSize");
  *limit = n;
  return HSUMMA_OK;
}

int launch_split_bf16(const GridPlan &g, int S, const void *As, const void *Bs, int32_t *D,
                      cudaStream_t s) {
  const int64_t Kpad = ceil_div(g.K, 64) * 64;
  const int a_box = (TM / 8) % g.cn == 0 ? TM / g.cn : 8;
  const int b_box = (TN / 8) % g.cm == 0 ? TN / g.cm : 8;
  const auto BF16 = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap tA, tB, tApf, tBpf;
  if (!encode_tmap_3d(&tA, BF16, 2, As, Kpad, g.M, S, BKS, a_box, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tB, BF16, 2, Bs, Kpad, g.N, S, BKS, b_box, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_3d(&tApf, BF16, 2, As, Kpad, g.M, S, BKS, TM, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_3d(&tBpf, BF16, 2, Bs, Kpad, g.N, S, BKS, TN, CU_TENSOR_MAP_SWIZZLE_NONE))
    return HSUMMA_ERR_ARG;
  SplitParams p;
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
  p.nkb = (int)(Kpad / BKS);
  p.nseg = split_planes(g.K, S, HSUMMA_BF16_SLICES);
  p.ch = bf16_chunk_products(slice_width(HSUMMA_BF16_SLICES, S)) / BKS;
  p.segst = kSegChunks * p.ch;
  p.counters = state().d_counters;
  p.status = state().d_status;
  const bool flat = g.cm * g.cn == 1;
  auto kern = g.cyc ? (flat ? bf16_diag_kernel<true, true> : bf16_diag_kernel<true, false>)
                    : (flat ? bf16_diag_kernel<false, true> : bf16_diag_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
  if (g.cm * g.cn > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(non-portable cluster)");
  }
  // one cluster per cluster tile (the kernel can also loop over tiles with a
  // smaller grid, but clusters resident together drift apart along k and then
  // share less in L2 than freshly launched ones)
  cudaLaunchConfig_t cfg = {};
  const int ntiles = (g.Q / g.cn) * (g.P / g.cm);
  cfg.gridDim = dim3((unsigned)(ntiles * g.cn), (unsigned)g.cm, 1);
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
  if (e != cudaSuccess) return cuda_fail(e, "launch bf16_diag_kernel");
  count_launch();
  return HSUMMA_OK;
}

}  // namespace hs
