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

// The digits of one value, slice by slice: Y_s = RN(|x| 2^-e 2^(w s)) (ties to
// even) as a signed integer, and digit s = Y_s - 2^w Y_(s-1).  The state holds
// the significand, the exponent of its last bit, the sign and Y_(s-1), so no
// table indexed by the (run-time) slice number is needed.
struct DigitGen {
  unsigned long long m;
  int lsb;    // binary exponent of m's least significant bit
  bool neg;
  long long prev;

  __device__ __forceinline__ void init(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    neg = (bits >> 63) != 0;
    const int E = (int)((bits >> 52) & 0x7FF);
    m = bits & 0xFFFFFFFFFFFFFull;
    if (E > 0) {
      m |= 1ull << 52;
      lsb = E - 1075;
    } else {
      lsb = -1074;
    }
    prev = 0;
  }

  // digit s (1-based) of w-bit slices for the scale 2^-e
  template <int W>
  __device__ __forceinline__ int next(int s, int e) {
    // |x| 2^-e 2^(w s) = m 2^sh, rounded to nearest (ties to even):
    // RNE(m / 2^d) = (m + 2^(d-1) - 1 + ((m >> d) & 1)) >> d for 1 <= d <= 54
    const int sh = lsb - e + W * s;
    unsigned long long y;
    if (sh >= 0) {
      // m 2^sh < 2^(w s - 1) <= 2^55 when e comes from the exponent scan (the
      // guard only keeps the shift defined for other e)
      y = m << (sh < 63 ? sh : 63);
    } else if (-sh > 54) {
      y = 0;        // m 2^sh < 2^53 2^-55 < 1/2
    } else {
      const int d = -sh;
      y = (m + ((1ull << (d - 1)) - 1ull) + ((m >> d) & 1ull)) >> d;
    }
    const long long Y = neg ? -(long long)y : (long long)y;
    const int t = (int)(Y - prev * (1ll << W));
    prev = Y;
    return t;
  }
};

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
      __nv_bfloat162 b = __floats2bfloat162_rn((float)t[2 * h], (float)t[2 * h + 1]);
      w[h] = *reinterpret_cast<uint32_t *>(&b);
    }
    *reinterpret_cast<uint4 *>(dst) = v;
  }
}

// A slices: As[s][i][k], k < Kp (zero beyond K); each thread 8 consecutive k
template <int KIND>
__global__ void __launch_bounds__(256) slices_rows_kernel(const double *__restrict__ A,
                                                          int64_t lda, int64_t M, int64_t K,
                                                          int64_t Kp,
                                                          const int32_t *__restrict__ e, int S,
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
  for (int u = 0; u < 8; ++u) g[u].init(x[u]);
  uint8_t *base = reinterpret_cast<uint8_t *>(out) + (i * Kp + k0) * EB;
  const int64_t plane = M * Kp * EB;
  for (int s = 1; s <= S; ++s) {
    int t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = g[u].next<W>(s, ei);
    store8<KIND>(base + (s - 1) * plane, t);
  }
}

// B slices, transposed: Bs[t][j][k]; a block transposes a 64 (k) x 64 (j) tile,
// each thread then forms 8 consecutive k of one column j (8 threads write one
// 64-k row segment of Bs)
template <int KIND>
__global__ void __launch_bounds__(256) slices_cols_kernel(const double *__restrict__ B,
                                                          int64_t ldb, int64_t K, int64_t N,
                                                          int64_t Kp,
                                                          const int32_t *__restrict__ f, int S,
                                                          void *__restrict__ out) {
  constexpr int W = KIND == HSUMMA_INT8_SLICES ? 7 : 8;
  constexpr int EB = KIND == HSUMMA_INT8_SLICES ? 1 : 2;
  __shared__ double tile[64][65];
  const int64_t k0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 64;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 256 threads: 64 x 4
  for (int r = ty; r < 64; r += 4) {
    const int64_t k = k0 + r, j = j0 + tx;
    tile[r][tx] = (k < K && j < N) ? B[k * ldb + j] : 0.0;
  }
  __syncthreads();
  const int64_t plane = N * Kp * EB;
  // thread -> (j = j0 + jj, k = k0 + kk .. kk + 7)
  for (int idx = threadIdx.x; idx < 64 * 8; idx += 256) {
    const int jj = idx >> 3, kk = (idx & 7) * 8;
    const int64_t j = j0 + jj;
    if (j >= N) continue;
    const int fj = f[j];
    DigitGen g[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) g[u].init(tile[kk + u][jj]);
    uint8_t *base = reinterpret_cast<uint8_t *>(out) + (j * Kp + k0 + kk) * EB;
    for (int s = 1; s <= S; ++s) {
      int t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = g[u].next<W>(s, fj);
      store8<KIND>(base + (s - 1) * plane, t);
    }
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
// stores of C when its row allows, element by element otherwise.
template <int W, int S>
__global__ void __launch_bounds__(256) recombine_kernel(const int32_t *__restrict__ D, int nseg,
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
  __int128 X[4] = {0, 0, 0, 0};
#pragma unroll
  for (int d = 2; d <= S + 1; ++d) {
    long long Dd[4] = {0, 0, 0, 0};   // the segment planes of a diagonal sum exactly in 64 bits
    for (int g = 0; g < nseg; ++g) {
      const int32_t *src = D + (int64_t)((d - 2) * nseg + g) * plane + off;
      if (vec) {
        const int4 v = __ldg(reinterpret_cast<const int4 *>(src));
        Dd[0] += v.x;
        Dd[1] += v.y;
        Dd[2] += v.z;
        Dd[3] += v.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < N) Dd[u] += __ldg(src + u);
      }
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

}  // namespace

int launch_split_exponents(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                           const double *B, int64_t ldb, int32_t *e, int32_t *f,
                           cudaStream_t s) {
  int *status = state().d_status;
  if (M > 0) {
    const int64_t blocks = ceil_div(M, 8);
    exponents_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, lda, M, K, e, status);
  }
  if (N > 0) {
    exponents_cols_kernel<<<(unsigned)ceil_div(N, 64), 256, 0, s>>>(B, ldb, K, N, f, status);
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
  if (nA > 0) {
    const unsigned blocks = (unsigned)ceil_div(nA, 256);
    if (kind == HSUMMA_INT8_SLICES)
      slices_rows_kernel<HSUMMA_INT8_SLICES><<<blocks, 256, 0, s>>>(A, lda, M, K, Kp, e, S, As);
    else
      slices_rows_kernel<HSUMMA_BF16_SLICES><<<blocks, 256, 0, s>>>(A, lda, M, K, Kp, e, S, As);
  }
  if (N > 0) {
    dim3 grid((unsigned)(Kp / 64), (unsigned)ceil_div(N, 64));
    if (kind == HSUMMA_INT8_SLICES)
      slices_cols_kernel<HSUMMA_INT8_SLICES><<<grid, 256, 0, s>>>(B, ldb, K, N, Kp, f, S, Bs);
    else
      slices_cols_kernel<HSUMMA_BF16_SLICES><<<grid, 256, 0, s>>>(B, ldb, K, N, Kp, f, S, Bs);
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
