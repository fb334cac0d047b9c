// Split-precision path, the steps around the tensor-core products:
//   1. exponent scan   e_i = ilogb(max_k |A_ik|) + 2, f_j over the columns of B
//   2. slicing         S digits per entry, t_s = RN(r 2^(w s)) - 2^w RN(r 2^(w(s-1))),
//                      r = a 2^-e (round half to even), as int8 (w = 7) or bf16 (w = 8)
//   4. recombination   C_ij = RN(2^(e_i+f_j) sum_d D_d,ij 2^(-w d)), exact sum in
//                      128-bit integers, rounded once to binary64
// All three work on the bit patterns with integer instructions: binary64
// arithmetic is the slowest unit of this GPU and is not needed for any of them.
// The digit formula is the closed form of the Ozaki splitting r <- r 2^w - rint(r 2^w)
// (the remainder recursion telescopes because shifting by the even integer
// 2^w t does not change a round-half-to-even decision).
#include <cuda_bf16.h>

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

// columns of B: a block covers 64 columns (32 lanes x 2), its 8 warps split k
__global__ void exponents_cols_kernel(const double *__restrict__ B, int64_t ldb, int64_t K,
                                      int64_t N, int32_t *__restrict__ f, int *status) {
  __shared__ unsigned long long part[8][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * 64 + 2 * lane;
  unsigned long long m0 = 0, m1 = 0;
  const bool pairs = ((reinterpret_cast<uintptr_t>(B) | (uintptr_t)(ldb * 8)) & 15) == 0;
  if (j0 + 1 < N && pairs) {
    for (int64_t k = warp; k < K; k += 8) {
      const double2 v = *reinterpret_cast<const double2 *>(B + k * ldb + j0);
      m0 = max(m0, absbits(v.x));
      m1 = max(m1, absbits(v.y));
    }
  } else {
    for (int64_t k = warp; k < K; k += 8) {
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
    const int64_t j = (int64_t)blockIdx.x * 64 + threadIdx.x;
    if (j < N) {
      bool nf = false;
      f[j] = exponent_from_bits(m, &nf);
      if (nf) record_error(status, HSUMMA_ERR_NONFINITE, kSiteNonFinite);
    }
  }
}

// The digits of one value, slice by slice.  With F = floor(|x| 2^-e 2^64)
// (below 2^63, since the exponent scan makes |x| 2^-e < 1/2) and Y_s =
// RN(|x| 2^-e 2^(W s)) (ties to even), digit s is t_s = Y_s - 2^W Y_(s-1).
// Writing Y_s = q_s + c_s with q_s = floor(F / 2^(p+1)), p = 63 - W s, and c_s
// the rounding increment, and since q_(s-1) = floor(q_s / 2^W):
//   t_s = (q_s mod 2^W) + c_s - 2^W c_(s-1),
// where q_s mod 2^W is the W-bit field of F above bit p and
//   c_s = (bit p of F) and (any lower bit of F, or a bit dropped below F,
//                           or bit p + 1 of F)          (round half to even).
// Bit p is the same for every value of a slice, so a digit costs a shift, a
// comparison, a few masks and no branch ("any lower bit" is tz < p, tz the
// trailing zero count of F, -1 when bits were dropped below F).  W S <= 63
// (bf16: S <= 7; int8: S <= 8).  A negative x has the negated digits
// (rounding to nearest is symmetric).
struct DigitGen {
  unsigned long long F;
  int tz;            // trailing zeros of F; -1 if |x| 2^-e 2^64 is not an integer; 64 if 0
  bool neg;
  int cprev;         // c_(s-1)

  __device__ __forceinline__ void init(double x, int e) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    neg = (bits >> 63) != 0;
    const int E = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    int lsb;        // binary exponent of m's least significant bit
    if (E > 0) {
      m |= 1ull << 52;
      lsb = E - 1075;
    } else {
      lsb = -1074;
    }
    const int sh = lsb - e + 64;     // |x| 2^-e 2^64 = m 2^sh
    bool sticky;                     // bits of m dropped below F
    if (sh >= 0) {
      F = m << (sh < 63 ? sh : 63);  // exact (the guard only keeps the shift defined)
      sticky = false;
    } else if (sh > -64) {
      F = m >> -sh;
      sticky = (m << (64 + sh)) != 0;
    } else {
      F = 0;
      sticky = m != 0;
    }
    tz = sticky ? -1 : (F ? __ffsll((long long)F) - 1 : 64);
    cprev = 0;
  }

  // digit s for p = 63 - W s (the same for every value)
  template <int W>
  __device__ __forceinline__ int next(int p) {
    const uint32_t win = (uint32_t)(F >> p);    // bit 0: rounding bit; bits 1..W: field
    const int field = (int)((win >> 1) & ((1u << W) - 1u));
    const int c = (int)(win & 1u) & ((int)(tz < p) | (field & 1));
    const int t = field + c - (cprev << W);
    cprev = c;
    return neg ? -t : t;
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
    uint2 v;
    v.x = (uint32_t)(uint8_t)t[0] | ((uint32_t)(uint8_t)t[1] << 8) |
          ((uint32_t)(uint8_t)t[2] << 16) | ((uint32_t)(uint8_t)t[3] << 24);
    v.y = (uint32_t)(uint8_t)t[4] | ((uint32_t)(uint8_t)t[5] << 8) |
          ((uint32_t)(uint8_t)t[6] << 16) | ((uint32_t)(uint8_t)t[7] << 24);
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

// A slices: As[s][i][k], k < Kp (zero beyond K); each thread 8 consecutive k.
// S is a template parameter so that every digit's bit position is a constant.
template <int KIND, int S>
__global__ void __launch_bounds__(256) slices_rows_kernel(const double *__restrict__ A,
                                                          int64_t lda, int64_t M, int64_t K,
                                                          int64_t Kp,
                                                          const int32_t *__restrict__ e,
                                                          void *__restrict__ out) {
  constexpr int W = KIND == HSUMMA_INT8_SLICES ? 7 : 8;
  constexpr int EB = KIND == HSUMMA_INT8_SLICES ? 1 : 2;
  const int64_t groups = Kp / 8;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= M * groups) return;
  const int64_t i = gid / groups, k0 = (gid % groups) * 8;
  const int ei = e[i];
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
  for (int u = 0; u < 8; ++u) g[u].init(x[u], ei);
  uint8_t *base = reinterpret_cast<uint8_t *>(out) + (i * Kp + k0) * EB;
  const int64_t plane = M * Kp * EB;
#pragma unroll
  for (int s = 1; s <= S; ++s) {
    int t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = g[u].next<W>(63 - W * s);
    store8<KIND>(base + (s - 1) * plane, t);
  }
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
  constexpr int W = KIND == HSUMMA_INT8_SLICES ? 7 : 8;
  constexpr int EB = KIND == HSUMMA_INT8_SLICES ? 1 : 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t njb = (uint32_t)((N + 31) / 32);
  const uint32_t kb = blockIdx.x / njb, jb = blockIdx.x - kb * njb;
  const int64_t j = (int64_t)jb * 32 + (w & 1) * 16 + (lane >> 1);
  const int64_t k0 = (int64_t)kb * 64 + (w >> 1) * 16 + (lane & 1) * 8;
  if (j >= N) return;
  const int fj = f[j];
  double x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = k0 + u < K ? B[(k0 + u) * ldb + j] : 0.0;
  DigitGen g[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) g[u].init(x[u], fj);
  uint8_t *base = reinterpret_cast<uint8_t *>(out) + (j * Kp + k0) * EB;
  const int64_t plane = N * Kp * EB;
#pragma unroll
  for (int s = 1; s <= S; ++s) {
    int t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = g[u].next<W>(63 - W * s);
    store8<KIND>(base + (s - 1) * plane, t);
  }
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

// The same for X that fits in 64 bits and a normal result (the common case):
// 64-bit integer work only; anything else goes to the general routine.
__device__ __forceinline__ double round_scaled(__int128 X, int k) {
  const long long lo = (long long)X;
  if ((__int128)lo == X && lo != 0) {
    const bool neg = lo < 0;
    const unsigned long long m = neg ? 0ull - (unsigned long long)lo : (unsigned long long)lo;
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
  return round_scaled_i128(X, k);
}

// X = sum_d D_d 2^(w (S+1-d)) by Horner's rule (constant shifts), rounded once.
// Each thread takes four consecutive columns of one row: 16-byte loads from
// every plane when the rows are 16-byte aligned (N a multiple of 4), 16-byte
// stores of C when its row allows, element by element otherwise.  The first
// segment plane of every diagonal is loaded before any arithmetic, so that
// all S loads of a thread are in flight at once; further segment planes (K
// beyond one segment) follow one diagonal at a time.
// (four resident blocks per SM keep more loads in flight; the kernels of 7 and
// 8 slices need more than the 64 registers that leaves)
template <int W, int S>
__global__ void __launch_bounds__(256, S <= 6 ? 4 : 3) recombine_kernel(const int32_t *__restrict__ D, int nseg,
                                                        int64_t M, int64_t N,
                                                        const int32_t *__restrict__ e,
                                                        const int32_t *__restrict__ f,
                                                        double *__restrict__ C, int64_t ldc) {
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
  __int128 X[4] = {0, 0, 0, 0};
#pragma unroll
  for (int d = 0; d < S; ++d) {
    long long Dd[4] = {first[d][0], first[d][1], first[d][2], first[d][3]};
    // the segment planes of a diagonal sum exactly in 64 bits
    for (int g = 1; g < nseg; ++g) {
      int v[4];
      load4(D + (int64_t)(d * nseg + g) * plane + off, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) Dd[u] += v[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) X[u] = (X[u] << W) + (__int128)Dd[u];
  }
  const int k = e[i] - W * (S + 1);
  double out[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) out[u] = j0 + u < N ? round_scaled(X[u], k + f[j0 + u]) : 0.0;
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

template <int W, int S>
void recombine_launch(dim3 grid, cudaStream_t s, const int32_t *D, int nseg, int64_t M,
                      int64_t N, const int32_t *e, const int32_t *f, double *C, int64_t ldc) {
  recombine_kernel<W, S><<<grid, 256, 0, s>>>(D, nseg, M, N, e, f, C, ldc);
  count_launch();
}

template <int W>
void recombine_dispatch(int S, dim3 grid, cudaStream_t s, const int32_t *D, int nseg,
                        int64_t M, int64_t N, const int32_t *e, const int32_t *f, double *C,
                        int64_t ldc) {
  switch (S) {
    case 1: recombine_launch<W, 1>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    case 2: recombine_launch<W, 2>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    case 3: recombine_launch<W, 3>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    case 4: recombine_launch<W, 4>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    case 5: recombine_launch<W, 5>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    case 6: recombine_launch<W, 6>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    case 7: recombine_launch<W, 7>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
    default: recombine_launch<W, 8>(grid, s, D, nseg, M, N, e, f, C, ldc); break;
  }
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
    exponents_cols_kernel<<<(unsigned)ceil_div(N, 64), 256, 0, s>>>(B, ldb, K, N, f, status);
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
  // one grid row per matrix row, in bands of at most 65535 rows; a band starts
  // r0 rows in: D, e and C advance by r0 rows, the plane stride stays M N
  for (int64_t r0 = 0; r0 < M; r0 += 65535) {
    const int64_t rows = (M - r0) < 65535 ? (M - r0) : 65535;
    dim3 grid((unsigned)ceil_div(ceil_div(N, 4), 256), (unsigned)rows);
    if (kind == HSUMMA_INT8_SLICES)
      recombine_dispatch<7>(S, grid, s, D + r0 * N, nseg, M, N, e + r0, f, C + r0 * ldc, ldc);
    else
      recombine_dispatch<8>(S, grid, s, D + r0 * N, nseg, M, N, e + r0, f, C + r0 * ldc, ldc);
  }
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? HSUMMA_OK : cuda_fail(err, "launch recombination");
}

}  // namespace hs
