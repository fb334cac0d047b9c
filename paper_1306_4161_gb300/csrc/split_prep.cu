// Split-precision path, the steps around the tensor-core products:
//   1. exponent scan   e_i = ilogb(max_k |A_ik|) + 2, f_j over the columns of B
//   2. slicing         S digits per entry, t_s = RN(r 2^(w s)) - 2^w RN(r 2^(w(s-1))),
//                      r = a 2^-e (round half to even), as int8 (w = 7) or bf16 (w = 9;
//                      8 for S = 7)
//   4. recombination   C_ij = RN(2^(e_i+f_j) sum_d D_d,ij 2^(-w d)), exact sum in
//                      128-bit integers, rounded once to binary64
// All three work on the bit patterns with integer instructions: binary64
// arithmetic is the slowest unit of this GPU and is not needed for any of them.
// The digit formula is the closed form of the Ozaki splitting r <- r 2^w - rint(r 2^w)
// (the remainder recursion telescopes because shifting by the even integer
// 2^w t does not change a round-half-to-even decision).
#include <cuda_bf16.h>

#include <cmath>

#include "internal.h"
#include "ptx.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

// max over |x| by bit pattern (non-negative doubles order like their bits)
__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// exponent e (ilogb + 2) from the largest |x| bit pattern; flags Inf/NaN
__device__ __forceinline__ int exponent_from_bits(unsigned long long b, bool *nonfinite) {
  const int E = (int)(b >> 52);
  if (E == 0x7FF) {
    *nonfinite = true;
    return 0;
  }
  if (b == 0) return 0;
  int ilogb;
  if (E > 0)
    ilogb = E - 1023;
  else
    ilogb = (63 - __clzll((long long)(b & 0xFFFFFFFFFFFFFull))) - 1074;
  return ilogb + 2;
}

// rows of A: one warp per row
__global__ void exponents_rows_kernel(const double *__restrict__ A, int64_t lda, int64_t M,
                                      int64_t K, int32_t *__restrict__ e, int *status) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const double *a = A + row * lda;
  unsigned long long m = 0;
  if ((reinterpret_cast<uintptr_t>(a) & 15) == 0) {
    // 16-byte aligned row: pairs
    const int64_t K2 = K & ~int64_t(1);
    for (int64_t k = 2 * lane; k < K2; k += 64) {
      const double2 v = *reinterpret_cast<const double2 *>(a + k);
      m = max(m, max(absbits(v.x), absbits(v.y)));
    }
    if ((K & 1) && lane == 0) m = max(m, absbits(a[K - 1]));
  } else {
    for (int64_t k = lane; k < K; k += 32) m = max(m, absbits(a[k]));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    bool nf = false;
    e[row] = exponent_from_bits(m, &nf);
    if (nf) record_error(status, HSUMMA_ERR_NONFINITE, kSiteNonFinite);
  }
}

// columns of B: a block covers 64 columns (32 lanes x 2) and one of the
// gridDim.y slices of k, its 8 warps splitting that slice; the gridDim.y blocks
// of a column group form one cluster (1 x gridDim.y), and its first CTA
// reduces their maxima through distributed shared memory.  Every thread
// reaches both cluster barriers.
__global__ void exponents_cols_kernel(const double *__restrict__ B, int64_t ldb, int64_t K,
                                      int64_t N, int32_t *__restrict__ f, int *status) {
  __shared__ unsigned long long part[8][64];
  __shared__ unsigned long long colmax[64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * 64 + 2 * lane;
  const int64_t kc = (K + gridDim.y - 1) / gridDim.y;
  const int64_t kb = (int64_t)blockIdx.y * kc, ke = kb + kc < K ? kb + kc : K;
  unsigned long long m0 = 0, m1 = 0;
  const bool pairs = ((reinterpret_cast<uintptr_t>(B) | (uintptr_t)(ldb * 8)) & 15) == 0;
  if (j0 + 1 < N && pairs) {
    for (int64_t k = kb + warp; k < ke; k += 8) {
      const double2 v = *reinterpret_cast<const double2 *>(B + k * ldb + j0);
      m0 = max(m0, absbits(v.x));
      m1 = max(m1, absbits(v.y));
    }
  } else {
    for (int64_t k = kb + warp; k < ke; k += 8) {
      if (j0 < N) m0 = max(m0, absbits(B[k * ldb + j0]));
      if (j0 + 1 < N) m1 = max(m1, absbits(B[k * ldb + j0 + 1]));
    }
  }
  part[warp][2 * lane] = m0;
  part[warp][2 * lane + 1] = m1;
  __syncthreads();
  if (threadIdx.x < 64) {
    unsigned long long m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m = max(m, part[w][threadIdx.x]);
    colmax[threadIdx.x] = m;
  }
  const bool split = gridDim.y > 1;
  if (split) cluster_sync();         // every CTA's colmax is written
  if (threadIdx.x < 64 && cluster_ctarank() == 0) {
    unsigned long long m = colmax[threadIdx.x];
    for (uint32_t r = 1; r < gridDim.y; ++r)
      m = max(m, ld_shared_cluster_u64(smem_u32(&colmax[threadIdx.x]), r));
    const int64_t j = (int64_t)blockIdx.x * 64 + threadIdx.x;
    if (j < N) {
      bool nf = false;
      f[j] = exponent_from_bits(m, &nf);
      if (nf) record_error(status, HSUMMA_ERR_NONFINITE, kSiteNonFinite);
    }
  }
  if (split) cluster_sync();         // the first CTA has read every colmax
}

// The digits of one value, slice by slice.  With F = floor(|x| 2^-e 2^64)
// (below 2^63, since the exponent scan makes |x| 2^-e < 1/2) and
// Y_s = RN(|x| 2^-e 2^(W s)) (ties to even), digit s is t_s = Y_s - 2^W Y_(s-1).
// Y_s is F / 2^(p+1), p = 63 - W s, rounded to nearest even; the bits below the
// rounding bit p only matter as "any of them set", so
//   Y_s = (F + 2^p - 1 + bit p+1 of F) >> (p + 1)
// provided that a bit dropped below F (a value far below the row's largest)
// still counts: it is or-ed into bit 0 of F, which is never a digit or rounding
// bit (p >= 7, since W S <= 56).  F is held as two 32-bit words Fh:Fl.  For
// p >= 33 the low word only matters as that same "any bit" flag, so it is folded
// into bit 0 of the high word (Fhs) and the digit takes one 32-bit add and shift;
// for p <= 31 the add runs over both words.  Y_s and 2^W Y_(s-1) are only needed
// modulo 2^32, since their difference is small.  A negative x has the negated
// digits (rounding to nearest is symmetric).  Bit p is the same for every value
// of a slice, so a digit costs a few integer instructions and no branch.
struct DigitGen {
  uint32_t Fh, Fl;   // F = Fh 2^32 + Fl, with dropped bits or-ed into bit 0 of Fl
  uint32_t Fhs;      // Fh with "Fl != 0" or-ed into bit 0
  uint32_t Yprev;    // Y_(s-1) modulo 2^32
  int sgn;           // +1 or -1

  // eb = e + 1011: then |x| 2^-e 2^64 = m 2^sh with sh = max(E, 1) - eb, for
  // the significand m (hidden bit included) and the biased exponent E of x.
  __device__ __forceinline__ void init(double x, int eb) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7FFu);
    const uint32_t mhi = (hi & 0xFFFFFu) | (E ? 0x100000u : 0u);
    const int sh = max(E, 1) - eb;
    sgn = ((int)hi >> 31) | 1;
    if ((unsigned)sh < 32u) {
      // every normal value of a finite row (sh <= 10): nothing is dropped
      Fh = __funnelshift_l(lo, mhi, (unsigned)sh);
      Fl = lo << sh;
    } else {
      const uint2 F = shift_rare(mhi, lo, sh);
      Fh = F.x;
      Fl = F.y;
    }
    Fhs = Fh | (Fl != 0u ? 1u : 0u);
    Yprev = 0u;
  }

  // sh < 0 (values more than 2^11 below the row's largest) or sh >= 32 (tiny
  // subnormals, whose significand then fits the low word; also whatever a
  // non-finite input gives, which the exponent scan has reported): returns
  // (Fh, Fl) with the dropped bits or-ed into bit 0 of Fl
  static __device__ __noinline__ uint2 shift_rare(uint32_t mhi, uint32_t lo, int sh) {
    uint32_t h, l, dropped;
    if (sh >= 32) {
      h = __funnelshift_lc(0u, lo, (unsigned)(sh - 32));    // lo << (sh - 32), 0 past 63
      l = 0u;
      dropped = 0u;
    } else if (sh > -32) {
      const unsigned r = (unsigned)(-sh);                   // 1..31
      h = mhi >> r;
      l = __funnelshift_r(lo, mhi, r);
      dropped = lo << (32u - r);
    } else if (sh > -64) {
      const unsigned r = (unsigned)(-sh) - 32u;             // 0..31
      h = 0u;
      l = mhi >> r;
      dropped = lo | __funnelshift_lc(0u, mhi, 32u - r);    // the low r bits of mhi
    } else {
      h = 0u;
      l = 0u;
      dropped = mhi | lo;
    }
    return make_uint2(h, l | (dropped != 0u ? 1u : 0u));
  }

  // the signed digit s (1-based); W S <= 56, so p = 63 - W s >= 7
  template <int W, int s>
  __device__ __forceinline__ int next() {
    constexpr int p = 63 - W * s;
    static_assert(p >= 7, "at most 56 digit bits");
    uint32_t Y;
    if constexpr (p >= 33) {
      constexpr int q = p - 32;
      Y = (Fhs + ((1u << q) - 1u) + ((Fhs >> (q + 1)) & 1u)) >> (q + 1);
    } else {
      const unsigned long long F = ((unsigned long long)Fh << 32) | Fl;
      Y = (uint32_t)((F + ((1ull << p) - 1ull) + ((F >> (p + 1)) & 1ull)) >> (p + 1));
    }
    const int t = (int)(Y - (Yprev << W));
    Yprev = Y;
    return t * sgn;
  }
};

// An integer |t| < 2^22 as a float without the integer-to-float unit: its bits
// placed in the significand of 2^23 + 2^22, then that constant subtracted.
__device__ __forceinline__ float small_int_to_float(int t) {
  return __int_as_float(0x4B400000 + t) - 12582912.0f;
}

// Eight digits of one slice, stored at dst: bf16 (16 bytes) or int8 (8 bytes).
template <int KIND>
__device__ __forceinline__ void store8(void *dst, const int (&t)[8]) {
  if (KIND == HSUMMA_INT8_SLICES) {
    // low bytes of t[0..3] (t[4..7]) by byte permutes: two pairs, then the pairs
    uint2 v;
    v.x = __byte_perm(__byte_perm(t[0], t[1], 0x0040), __byte_perm(t[2], t[3], 0x0040), 0x5410);
    v.y = __byte_perm(__byte_perm(t[4], t[5], 0x0040), __byte_perm(t[6], t[7], 0x0040), 0x5410);
    *reinterpret_cast<uint2 *>(dst) = v;
  } else {
    uint4 v;
    uint32_t *w = reinterpret_cast<uint32_t *>(&v);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      __nv_bfloat162 b =
          __floats2bfloat162_rn(small_int_to_float(t[2 * h]), small_int_to_float(t[2 * h + 1]));
      w[h] = *reinterpret_cast<uint32_t *>(&b);
    }
    *reinterpret_cast<uint4 *>(dst) = v;
  }
}

// Slices s..S of eight values, slice s at base + (s - 1) plane (the slice
// index is a template argument, so each digit's bit position is a constant).
template <int KIND, int W, int s, int S>
__device__ __forceinline__ void store_digits(DigitGen (&g)[8], uint8_t *base, int64_t plane) {
  if constexpr (s <= S) {
    int t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = g[u].template next<W, s>();
    store8<KIND>(base + (s - 1) * plane, t);
    store_digits<KIND, W, s + 1, S>(g, base, plane);
  }
}

// A slices: As[s][i][k], k < Kp (zero beyond K); each thread 8 consecutive k.
// S is a template parameter so that every digit's bit position is a constant.
template <int KIND, int S>
__global__ void __launch_bounds__(256) slices_rows_kernel(const double *__restrict__ A,
                                                          int64_t lda, int64_t M, int64_t K,
                                                          int64_t Kp,
                                                          const int32_t *__restrict__ e,
                                                          void *__restrict__ out) {
  constexpr int W = slice_width(KIND, S);
  constexpr int EB = KIND == HSUMMA_INT8_SLICES ? 1 : 2;
  const int64_t groups = Kp / 8;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= M * groups) return;
  const int64_t i = gid / groups, k0 = (gid % groups) * 8;
  const int eb = e[i] + 1011;
  double x[8];
  const double *a = A + i * lda + k0;
  if (k0 + 7 < K && (reinterpret_cast<uintptr_t>(a) & 15) == 0) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 v = reinterpret_cast<const double2 *>(a)[h];
      x[2 * h] = v.x;
      x[2 * h + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = k0 + u < K ? a[u] : 0.0;
  }
  DigitGen g[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) g[u].init(x[u], eb);
  uint8_t *base = reinterpret_cast<uint8_t *>(out) + (i * Kp + k0) * EB;
  store_digits<KIND, W, 1, S>(g, base, M * Kp * EB);
}

// B slices, transposed: Bs[t][j][k].  A block covers 32 columns x 64 k; warp
// w takes 16 columns (w & 1) and 16 k (w >> 1), and lanes 2i and 2i + 1 take
// k .. k + 7 and k + 8 .. k + 15 of one column, so that a warp's store of a
// slice fills 16 whole 32-byte sectors (bf16) and its loads read 16
// consecutive doubles of each of 16 rows of B.  One-dimensional grid, column
// blocks fastest (neighbouring blocks read the same rows of B); any product
// whose slices fit in memory has fewer than 2^31 blocks.
template <int KIND, int S>
__global__ void __launch_bounds__(256) slices_cols_kernel(const double *__restrict__ B,
                                                          int64_t ldb, int64_t K, int64_t N,
                                                          int64_t Kp,
                                                          const int32_t *__restrict__ f,
                                                          void *__restrict__ out) {
  constexpr int W = slice_width(KIND, S);
  constexpr int EB = KIND == HSUMMA_INT8_SLICES ? 1 : 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t njb = (uint32_t)((N + 31) / 32);
  const uint32_t kb = blockIdx.x / njb, jb = blockIdx.x - kb * njb;
  const int64_t j = (int64_t)jb * 32 + (w & 1) * 16 + (lane >> 1);
  const int64_t k0 = (int64_t)kb * 64 + (w >> 1) * 16 + (lane & 1) * 8;
  if (j >= N) return;
  const int eb = f[j] + 1011;
  double x[8];
  const double *b = B + k0 * ldb + j;
  if (k0 + 7 < K) {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = __ldg(b + u * ldb);
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = k0 + u < K ? __ldg(b + u * ldb) : 0.0;
  }
  DigitGen g[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) g[u].init(x[u], eb);
  uint8_t *base = reinterpret_cast<uint8_t *>(out) + (j * Kp + k0) * EB;
  store_digits<KIND, W, 1, S>(g, base, N * Kp * EB);
}

// RN(X 2^k) for a 128-bit integer X, ties to even, subnormals and overflow
// handled: the value is rounded once, at the precision its exponent allows.
__device__ __noinline__ double round_scaled_i128(__int128 X, int k) {
  if (X == 0) return 0.0;
  const bool neg = X < 0;
  unsigned __int128 m = neg ? (unsigned __int128)(-X) : (unsigned __int128)X;
  const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
  const int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  const int e = nb - 1 + k;               // exponent of the leading bit
  int ulp = e - 52;                       // exponent of the last kept bit
  if (ulp < -1074) ulp = -1074;
  const int drop = ulp - k;               // low bits of m below the last kept bit
  unsigned long long q;
  if (drop <= 0) {
    q = (unsigned long long)(m << (-drop));   // < 2^53
  } else if (drop > nb) {
    q = 0;                                  // below half of the smallest step
  } else {
    const unsigned __int128 qq = m >> drop;
    const unsigned __int128 rem = m - (qq << drop);
    const unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
    q = (unsigned long long)qq;
    if (rem > half || (rem == half && (q & 1ull))) q += 1;
  }
  if (q == (1ull << 53)) {                 // rounding carried into a new binade
    q >>= 1;
    ulp += 1;
  }
  unsigned long long bits;
  if (q < (1ull << 52)) {
    bits = q;                               // subnormal (ulp == -1074) or zero
  } else {
    const long long biased = (long long)ulp + 1075;
    if (biased >= 2047)
      bits = 0x7FF0000000000000ull;         // overflow rounds to infinity
    else
      bits = ((unsigned long long)biased << 52) | (q & 0xFFFFFFFFFFFFFull);
  }
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double((long long)bits);
}

// The same for a 64-bit X: 64-bit integer work when the result is normal (the
// common case); anything else goes to the general routine.
__device__ __forceinline__ double round_scaled64(long long X, int k) {
  if (X != 0) {
    const bool neg = X < 0;
    const unsigned long long m = neg ? 0ull - (unsigned long long)X : (unsigned long long)X;
    const int nb = 64 - __clzll((long long)m);
    const int drop = nb - 53;
    unsigned long long q;
    int ulp;
    if (drop <= 0) {
      q = m << (-drop);
      ulp = k + drop;
    } else {
      q = (m + ((1ull << (drop - 1)) - 1ull) + ((m >> drop) & 1ull)) >> drop;
      ulp = k + drop;
      if (q == (1ull << 53)) {
        q >>= 1;
        ulp += 1;
      }
    }
    const int biased = ulp + 1075;
    if (biased >= 1 && biased <= 2046) {
      const unsigned long long bits = ((unsigned long long)biased << 52) |
                                      (q & 0xFFFFFFFFFFFFFull) |
                                      (neg ? 0x8000000000000000ull : 0ull);
      return __longlong_as_double((long long)bits);
    }
  }
  return round_scaled_i128((__int128)X, k);
}

__device__ __forceinline__ double round_scaled(__int128 X, int k) {
  const long long lo = (long long)X;
  if ((__int128)lo == X) return round_scaled64(lo, k);
  return round_scaled_i128(X, k);
}

// X = sum_d D_d 2^(w (S+1-d)) by Horner's rule (constant shifts), rounded once.
// Each thread takes four consecutive columns of one row: 16-byte loads from
// every plane when the rows are 16-byte aligned (N a multiple of 4), 16-byte
// stores of C when its row allows, element by element otherwise.  The first
// segment plane of every diagonal is loaded before any arithmetic, so that
// all S loads of a thread are in flight at once; a diagonal's further segment
// planes (np.n[d] of them in all; the planes past those hold zeros and are
// not read) are added in 64 bits.
// X fits in 64 bits whenever |D_2| <= T2: the host derives T2 from the range
// of the other diagonals (np.n[d] int32 planes each), so that
// |D_2| 2^(w (S-1)) + sum_(d>2) n_d 2^31 2^(w (S+1-d)) < 2^63 (every partial
// sum of Horner's rule is bounded by the same sum).  The diagonal sums the
// products give are far inside that bound; other values take the 128-bit path.
// (four resident blocks per SM keep more loads in flight; the kernels of 6 to
// 8 slices need more than the 64 registers that leaves)
struct DiagPlanes {
  int n[8];   // segment planes of diagonal d + 2 that the products can fill
};

template <int W, int S>
__global__ void __launch_bounds__(256, S <= 5 ? 4 : 3) recombine_kernel(const int32_t *__restrict__ D, int nseg,
                                                        DiagPlanes np, int64_t M, int64_t N,
                                                        const int32_t *__restrict__ e,
                                                        const int32_t *__restrict__ f,
                                                        double *__restrict__ C, int64_t ldc,
                                                        int64_t T2) {
  const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const int64_t i = blockIdx.y;
  if (j0 >= N) return;
  const int64_t plane = M * N, off = i * N + j0;
  const bool full = j0 + 3 < N;
  const bool vec = full && (N & 3) == 0;
  auto load4 = [&](const int32_t *src, int (&v)[4]) {
    if (vec) {
      const int4 q = __ldg(reinterpret_cast<const int4 *>(src));
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = j0 + u < N ? __ldg(src + u) : 0;
    }
  };
  int first[S][4];
#pragma unroll
  for (int d = 0; d < S; ++d) load4(D + (int64_t)(d * nseg) * plane + off, first[d]);
  // D_2 whole (its further planes, if any), which decides the width
  long long D2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) D2[u] = first[0][u];
  for (int g = 1; g < np.n[0]; ++g) {
    int v[4];
    load4(D + (int64_t)g * plane + off, v);
#pragma unroll
    for (int u = 0; u < 4; ++u) D2[u] += v[u];
  }
  int gmax = 1;
#pragma unroll
  for (int d = 1; d < S; ++d) gmax = np.n[d] > gmax ? np.n[d] : gmax;
  // X is linear in the planes: Horner's rule over the first planes, then each
  // further round g adds sum_(d>2) plane_g(D_d) 2^(w (S+1-d)), the round's
  // loads all in flight together (every partial sum is bounded as X is)
  auto round_g = [&](int g, int (&v)[S][4]) {
#pragma unroll
    for (int d = 1; d < S; ++d) {
      if (g < np.n[d]) {
        load4(D + (int64_t)(d * nseg + g) * plane + off, v[d]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[d][u] = 0;
      }
    }
  };
  const int k = e[i] - W * (S + 1);
  double out[4];
  bool narrow = true;
#pragma unroll
  for (int u = 0; u < 4; ++u) narrow = narrow && llabs(D2[u]) <= T2;
  if (narrow) {
    unsigned long long X[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      X[u] = (unsigned long long)D2[u];
#pragma unroll
      for (int d = 1; d < S; ++d) X[u] = (X[u] << W) + (unsigned long long)(long long)first[d][u];
    }
    for (int g = 1; g < gmax; ++g) {
      int v[S][4];
      round_g(g, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        unsigned long long Y = 0;
#pragma unroll
        for (int d = 1; d < S; ++d) Y = (Y << W) + (unsigned long long)(long long)v[d][u];
        X[u] += Y;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      out[u] = j0 + u < N ? round_scaled64((long long)X[u], k + f[j0 + u]) : 0.0;
  } else {
    __int128 X[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      X[u] = D2[u];
#pragma unroll
      for (int d = 1; d < S; ++d) X[u] = (X[u] << W) + (__int128)first[d][u];
    }
    for (int g = 1; g < gmax; ++g) {
      int v[S][4];
      round_g(g, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        __int128 Y = 0;
#pragma unroll
        for (int d = 1; d < S; ++d) Y = (Y << W) + (__int128)v[d][u];
        X[u] += Y;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = j0 + u < N ? round_scaled(X[u], k + f[j0 + u]) : 0.0;
  }
  double *dst = C + i * ldc + j0;
  if (full && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    reinterpret_cast<double2 *>(dst)[0] = make_double2(out[0], out[1]);
    reinterpret_cast<double2 *>(dst)[1] = make_double2(out[2], out[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (j0 + u < N) dst[u] = out[u];
  }
}

// T2 of the kernel above: the largest |D_2| for which X stays below 2^63 when
// every other diagonal d holds any sum of np.n[d-2] int32 planes; 2^31 admits
// every int32 plane, and -1 admits none (the other diagonals alone can pass
// 2^63: bf16 with S = 6).
int64_t recombine_narrow_bound(int W, int S, const DiagPlanes &np) {
  long double rest = 0.0L;
  for (int d = 3; d <= S + 1; ++d)
    rest += np.n[d - 2] * ldexpl(2147483648.0L, W * (S + 1 - d));
  const long double room = ldexpl(1.0L, 63) - 1.0L - rest;
  if (room < 0.0L) return -1;
  const long double t = floorl(room / ldexpl(1.0L, W * (S - 1)));
  return t >= 9.0e18L ? (int64_t)9000000000000000000LL : (int64_t)t;
}

template <int W, int S>
void recombine_launch(dim3 grid, cudaStream_t s, const int32_t *D, int nseg, const DiagPlanes &np,
                      int64_t M, int64_t N, const int32_t *e, const int32_t *f, double *C,
                      int64_t ldc) {
  const int64_t T2 = recombine_narrow_bound(W, S, np);
  recombine_kernel<W, S><<<grid, 256, 0, s>>>(D, nseg, np, M, N, e, f, C, ldc, T2);
  count_launch();
}

// the slice count as a template argument; the width follows from kind and S
template <int KIND>
void recombine_dispatch(int S, dim3 grid, cudaStream_t s, const int32_t *D, int nseg,
                        const DiagPlanes &np, int64_t M, int64_t N, const int32_t *e,
                        const int32_t *f, double *C, int64_t ldc) {
#define HS_RECOMBINE(SS)                                                                    \
  recombine_launch<slice_width(KIND, SS), SS>(grid, s, D, nseg, np, M, N, e, f, C, ldc); \
  break
  switch (S) {
    case 1: HS_RECOMBINE(1);
    case 2: HS_RECOMBINE(2);
    case 3: HS_RECOMBINE(3);
    case 4: HS_RECOMBINE(4);
    case 5: HS_RECOMBINE(5);
    case 6: HS_RECOMBINE(6);
    case 7: HS_RECOMBINE(7);
    default: HS_RECOMBINE(8);
  }
#undef HS_RECOMBINE
}

// One slicing launch with the slice count as a template argument: rows of A
// (ROWS) or columns of B; X is the operand, L its leading dimension, R its
// rows (A) or columns (B), x the exponents.
template <int KIND, bool ROWS, int S>
void slices_launch(unsigned grid, cudaStream_t s, const double *X, int64_t L, int64_t R,
                   int64_t K, int64_t Kp, const int32_t *x, void *out) {
  if (ROWS)
    slices_rows_kernel<KIND, S><<<grid, 256, 0, s>>>(X, L, R, K, Kp, x, out);
  else
    slices_cols_kernel<KIND, S><<<grid, 256, 0, s>>>(X, L, K, R, Kp, x, out);
}

template <int KIND, bool ROWS>
void slices_dispatch(int S, unsigned grid, cudaStream_t s, const double *X, int64_t L,
                     int64_t R, int64_t K, int64_t Kp, const int32_t *x, void *out) {
  switch (S) {
    case 1: slices_launch<KIND, ROWS, 1>(grid, s, X, L, R, K, Kp, x, out); break;
    case 2: slices_launch<KIND, ROWS, 2>(grid, s, X, L, R, K, Kp, x, out); break;
    case 3: slices_launch<KIND, ROWS, 3>(grid, s, X, L, R, K, Kp, x, out); break;
    case 4: slices_launch<KIND, ROWS, 4>(grid, s, X, L, R, K, Kp, x, out); break;
    case 5: slices_launch<KIND, ROWS, 5>(grid, s, X, L, R, K, Kp, x, out); break;
    case 6: slices_launch<KIND, ROWS, 6>(grid, s, X, L, R, K, Kp, x, out); break;
    case 7: slices_launch<KIND, ROWS, 7>(grid, s, X, L, R, K, Kp, x, out); break;
    default:
      // 8 slices exist for int8 only (W S <= 63; bf16 stops at 7)
      if constexpr (KIND == HSUMMA_INT8_SLICES)
        slices_launch<KIND, ROWS, 8>(grid, s, X, L, R, K, Kp, x, out);
      break;
  }
}

}  // namespace

int launch_split_exponents(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                           const double *B, int64_t ldb, int32_t *e, int32_t *f,
                           cudaStream_t s) {
  int *status = state().d_status;
  if (M > 0) {
    const int64_t blocks = ceil_div(M, 8);
    exponents_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, lda, M, K, e, status);
    count_launch();
  }
  if (N > 0) {
    // k split over a cluster of up to 8 CTAs per column group, enough for
    // about four CTAs per SM (152 SMs) when N is small
    const int64_t nbx = ceil_div(N, 64);
    int ks = (int)ceil_div(4 * 152, nbx);
    ks = ks < 1 ? 1 : (ks > 8 ? 8 : ks);
    if (ks > K) ks = K > 1 ? (int)K : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nbx, (unsigned)ks, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)ks;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e2 = cudaLaunchKernelEx(&cfg, exponents_cols_kernel, B, ldb, K, N, f, status);
    if (e2 != cudaSuccess) return cuda_fail(e2, "launch exponent scan (columns)");
    count_launch();
  }
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? HSUMMA_OK : cuda_fail(err, "launch exponent scan");
}

int launch_split_slices(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                        const double *B, int64_t ldb, const int32_t *e, const int32_t *f,
                        int kind, int S, void *As, void *Bs, cudaStream_t s) {
  const int64_t Kp = ceil_div(K, 64) * 64;
  if (Kp == 0) return HSUMMA_OK;
  const int64_t nA = M * (Kp / 8);
  const int64_t ncb = N > 0 ? (Kp / 64) * ceil_div(N, 32) : 0;
  if (ceil_div(nA, 256) > 0x7fffffff || ncb > 0x7fffffff) {
    set_error("slicing grid too large (M=%lld N=%lld K=%lld)", (long long)M, (long long)N,
              (long long)K);
    return HSUMMA_ERR_UNSUPPORTED;
  }
  if (nA > 0) {
    const unsigned blocks = (unsigned)ceil_div(nA, 256);
    if (kind == HSUMMA_INT8_SLICES)
      slices_dispatch<HSUMMA_INT8_SLICES, true>(S, blocks, s, A, lda, M, K, Kp, e, As);
    else
      slices_dispatch<HSUMMA_BF16_SLICES, true>(S, blocks, s, A, lda, M, K, Kp, e, As);
    count_launch();
  }
  if (N > 0) {
    const unsigned grid = (unsigned)ncb;
    if (kind == HSUMMA_INT8_SLICES)
      slices_dispatch<HSUMMA_INT8_SLICES, false>(S, grid, s, B, ldb, N, K, Kp, f, Bs);
    else
      slices_dispatch<HSUMMA_BF16_SLICES, false>(S, grid, s, B, ldb, N, K, Kp, f, Bs);
    count_launch();
  }
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? HSUMMA_OK : cuda_fail(err, "launch slicing");
}

int launch_split_recombine(int64_t M, int64_t N, int64_t K, int kind, int S, const int32_t *D,
                           const int32_t *e, const int32_t *f, double *C, int64_t ldc,
                           cudaStream_t s) {
  const int nseg = split_planes(K, S, kind);
  DiagPlanes np = {};
  for (int d = 2; d <= S + 1 && d - 2 < 8; ++d)
    np.n[d - 2] = split_diagonal_planes(K, S, kind, d - 1);
  // one grid row per matrix row, in bands of at most 65535 rows; a band starts
  // r0 rows in: D, e and C advance by r0 rows, the plane stride stays M N
  for (int64_t r0 = 0; r0 < M; r0 += 65535) {
    const int64_t rows = (M - r0) < 65535 ? (M - r0) : 65535;
    dim3 grid((unsigned)ceil_div(ceil_div(N, 4), 256), (unsigned)rows);
    if (kind == HSUMMA_INT8_SLICES)
      recombine_dispatch<HSUMMA_INT8_SLICES>(S, grid, s, D + r0 * N, nseg, np, M, N, e + r0, f,
                                             C + r0 * ldc, ldc);
    else
      recombine_dispatch<HSUMMA_BF16_SLICES>(S, grid, s, D + r0 * N, nseg, np, M, N, e + r0, f,
                                             C + r0 * ldc, ldc);
  }
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? HSUMMA_OK : cuda_fail(err, "launch recombination");
}

}  // namespace hs
