// Host-side declarations shared by the translation units of libhsumma.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

namespace hs {

// Result of the host-side group resolution (Section III) and its realisation.
struct GridPlan {
  int64_t M, N, K;
  int P, Q, G, I, J;
  int cm, cn;            // realised cluster: rows x cols of CTAs (1 x 1 = flat)
  int64_t Mt, Nt;        // block sizes ceil(M/P), ceil(N/Q)
  int64_t Kq, Kp;        // ceil(K/Q), ceil(K/P): owner ranges of outer panels
  int nsub_m, nsub_n;    // sub-tiles per block
  int b, Bo;             // inner / outer panel widths
  bool cyc;              // block-cyclic layout (sub-tiles dealt round robin), else
                         // block-checkerboard (one block per processor)
};

// Row and column blocks of the pipelined host-buffer product (at most), and
// the timing events of its timeline: a start event, then a start and an end
// for each of its Cb + R + 2 R Cb phases (the copies of B_c in, of A_r in,
// then per block the product and the copy of C_rc out).
constexpr int kMaxHostBlocks = 4;      // row blocks
constexpr int kMaxHostColBlocks = 2;   // column blocks
constexpr int kMaxHostPhases =
    kMaxHostColBlocks + kMaxHostBlocks + 2 * kMaxHostBlocks * kMaxHostColBlocks;
constexpr int kHostTimelineEvents = 1 + 2 * kMaxHostPhases;

struct DeviceState {
  int device = -1;
  int sm_count = 0;
  int cluster_limit = 16;
  unsigned long long *d_counters = nullptr;  // 8 x u64
  int *d_status = nullptr;                   // 4 x int
  void *workspace = nullptr;
  size_t workspace_bytes = 0;
  void *host_staging = nullptr;              // device buffers of hsumma_gemm_host
  size_t host_staging_bytes = 0;
  bool bf16_pair = false;                    // bf16 products of 2 x 1 groups on CTA pairs
  int pair_launch = 0;                       // launch policy of the pair kernel (HSUMMA_PAIR_*)
  int pair_resident[3] = {0, 0, 0};          // resident clusters of CN pairs (0: not queried)
  void *tune_buf = nullptr;                  // model scoring inputs of hsumma_choose
  size_t tune_bytes = 0;
  cudaStream_t copy_in = nullptr;            // hsumma_gemm_host's copy streams
  cudaStream_t copy_out = nullptr;
  // hsumma_gemm_host's pipeline events, created once: ordering events (no
  // timing) and, when stage timing is on, timing events around every phase
  cudaEvent_t pipe_ev[3 + kMaxHostColBlocks + kMaxHostBlocks +
                      kMaxHostBlocks * kMaxHostColBlocks] = {};
  cudaEvent_t pipe_tev[kHostTimelineEvents] = {};
  int timeline_phases = 0;                   // phases the last timed call recorded
  int timeline_rows = 0, timeline_cols = 0;  // and its row and column blocks
  int host_row_blocks = 0;                   // row blocks of the last pipelined call
  int64_t host_row0[kMaxHostBlocks] = {};    // and the first row of each
};

DeviceState &state();
// Kernel launches issued on the product path (hsumma_launches reads the total).
void count_launch(int n = 1);
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// Tensor-map encoding through the driver entry point (no link to libcuda).
bool encode_tmap_2d(CUtensorMap *out, CUtensorMapDataType dtype, int elem_bytes,
                    const void *base, uint64_t inner, uint64_t outer,
                    uint64_t row_stride_elems, uint32_t box_inner, uint32_t box_outer,
                    CUtensorMapSwizzle swizzle);

// 3-D view {inner, rows, planes} of a planes x rows x inner array (row-major).
bool encode_tmap_3d(CUtensorMap *out, CUtensorMapDataType dtype, int elem_bytes,
                    const void *base, uint64_t inner, uint64_t rows, uint64_t planes,
                    uint32_t box_inner, uint32_t box_rows, CUtensorMapSwizzle swizzle);

// k-panel view of a slice tensor (S x rows x Kp, row-major, Kp a multiple of
// 64): 4-D {64, rows, Kp / 64, S} with strides {Kp, 64, rows Kp} elements, so
// that one box {64, box_rows, kz, 1} copies kz consecutive 64-column panels of
// box_rows rows at once (128-byte swizzle, 2-byte elements).
bool encode_tmap_kpanels(CUtensorMap *out, CUtensorMapDataType dtype, int elem_bytes,
                         const void *base, uint64_t Kp, uint64_t rows, uint64_t planes,
                         uint32_t box_rows, uint32_t kz);

// Launchers (return an hsumma_status).
int launch_fp64_hsumma(const GridPlan &g, const double *A, int64_t lda, const double *B,
                       int64_t ldb, double *C, int64_t ldc, cudaStream_t s);
int fp64_cluster_limit(int *limit);

int launch_split_exponents(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                           const double *B, int64_t ldb, int32_t *e, int32_t *f,
                           cudaStream_t s);
int launch_split_slices(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                        const double *B, int64_t ldb, const int32_t *e,
                        const int32_t *f, int kind, int S, void *As, void *Bs,
                        cudaStream_t s);
// Slice width w (bits) of S slices of a kind: the widest whose digits
// (|t| <= 2^(w-1)) the slice type holds exactly -- int8 7 (digits in
// [-64, 64]), bf16 9 (every integer of magnitude <= 256 is exact in bfloat16)
// -- capped so that w S <= 56 (the digit extraction works from a 64-bit fixed
// point image of each scaled value): bf16 with 7 slices takes 8.
constexpr int kMaxSlicedBits = 56;
__host__ __device__ constexpr int slice_width(int kind, int S) {
  return kind == 1 ? 7 : (S > 0 && 9 * S > kMaxSlicedBits ? kMaxSlicedBits / S : 9);
}
// bf16 digit products are integers of magnitude <= 2^(2w-2); an fp32
// accumulator stays exact (an integer <= 2^24) over 2^(26-2w) of them: 256
// products for w = 9, 1024 for w = 8.  The bf16 kernels drain their
// accumulators into int32 after at most that many ("chunk").
__host__ __device__ constexpr int bf16_chunk_products(int w) { return 1 << (26 - 2 * w); }
// Exact diagonal sums are stored as int32 planes D[d-2][seg][M][N]: a diagonal's
// sum over its (d-1) K products is cut into segments whose partial sums stay
// below 2^31 (bf16: 127 chunks, each summing to at most 2^24 in magnitude;
// int8: 2^18 products of magnitude <= 2^12 per segment).  The product kernels
// step through k in stages of at most 128 columns, a pair's last stage padded
// to 128, so diagonal d (d - 1 pairs) spans (d - 1) ceil(Kp / 128) 128-column
// stages; the plane count covers the longest (S pairs), and every kernel
// writes every plane of every diagonal (zeros past the diagonal's own
// segments).
constexpr int kSegChunks = 127;
inline int64_t split_segment_products(int S, int kind) {
  return kind == 1 ? (int64_t)1 << 18
                   : (int64_t)kSegChunks * bf16_chunk_products(slice_width(kind, S));
}
// the segments of a diagonal whose sum spans `pairs` slice pairs
inline int split_diagonal_planes(int64_t K, int S, int kind, int pairs) {
  const int64_t Kp = (K + 63) / 64 * 64;
  const int64_t K128 = (Kp + 127) / 128 * 128;
  const int64_t per_seg = split_segment_products(S, kind);
  const int64_t n = ((int64_t)pairs * K128 + per_seg - 1) / per_seg;
  return n < 1 ? 1 : (int)n;
}
inline int split_planes(int64_t K, int S, int kind = 2) {
  return split_diagonal_planes(K, S, kind, S);   // the longest diagonal: S pairs
}
int launch_split_bf16(const GridPlan &g, int S, const void *As, const void *Bs, int32_t *D,
                      cudaStream_t s);
int launch_split_int8(const GridPlan &g, int S, const void *As, const void *Bs, int32_t *D,
                      cudaStream_t s);
int launch_split_bf16_pair(const GridPlan &g, int S, const void *As, const void *Bs,
                           int32_t *D, cudaStream_t s);
int bf16_cluster_limit(int *limit);
// Clusters of the CTA-pair kernel (CN = 1: 2 x 1 groups, 2: 2 x 2) resident
// on the device at once.
int pair_resident_clusters(int CN, int *clusters);
int int8_cluster_limit(int *limit);
int launch_split_recombine(int64_t M, int64_t N, int64_t K, int kind, int S, const int32_t *D,
                           const int32_t *e, const int32_t *f, double *C, int64_t ldc,
                           cudaStream_t s);

int run_peak(int kind, int64_t work, double *rate);

// Learned cost model (mlp.cu): the parameters and feature standardisation
// loaded by hsumma_mlp_load (host copies; nullptr when none is loaded), and the
// bf16 scoring + argmin of n standardised feature rows on the device.
constexpr int kModelParams = 9089, kModelFeatures = 10;
const float *loaded_model(float *mean, float *stdv);
int mlp_pick_device(int n, const float *d_theta, const float *d_X, float *d_pred,
                    int32_t *d_best, cudaStream_t s);
// Automatic configuration (autotune.cu): forget every cached choice.
void forget_choices();
// drops the trained range of the cost model (a new model, or none, is loaded)
void forget_model_range();
// Drop the cached device addresses of hsumma_mlp_backward_noalloc's scratch
// (mlp.cu): they are looked up again on the next call on each device.
void forget_noalloc_scratch();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace hs
