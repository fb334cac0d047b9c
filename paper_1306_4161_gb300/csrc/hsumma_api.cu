// C ABI of libhsumma: argument checks, group resolution (Section III), the
// choice of kernels, the device error word, counters and workspace.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <array>
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/hsumma.h"
#include "internal.h"

namespace hs {

namespace {
thread_local char g_err[512] = "";
std::mutex g_mu;
DeviceState g_state;
bool g_init = false;

// Stage timing (hsumma_stage_timing): five events per recorded hsumma_gemm
// call, around exponent scan, slicing, products, recombination.
std::mutex g_stage_mu;
bool g_stage_on = false;
std::vector<std::array<cudaEvent_t, 5>> g_stage_ev;
size_t g_stage_used = 0;

// Events for the next recorded call, or nullptr when timing is off.
static cudaEvent_t *stage_slot() {
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (!g_stage_on) return nullptr;
  if (g_stage_used == g_stage_ev.size()) {
    std::array<cudaEvent_t, 5> ev;
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_stage_ev.push_back(ev);
  }
  return g_stage_ev[g_stage_used++].data();
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
}  // namespace

DeviceState &state() { return g_state; }

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return HSUMMA_ERR_CUDA;
}

bool encode_tmap_2d(CUtensorMap *out, CUtensorMapDataType dtype, int elem_bytes,
                    const void *base, uint64_t inner, uint64_t outer,
                    uint64_t row_stride_elems, uint32_t box_inner, uint32_t box_outer,
                    CUtensorMapSwizzle swizzle) {
  if (!g_encode) {
    set_error("tensor-map encoder unavailable (hsumma_init not called?)");
    return false;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_stride_elems * (uint64_t)elem_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(out, dtype, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): dims %llu x %llu, stride %llu B, box %u x %u",
              (int)r, (unsigned long long)inner, (unsigned long long)outer,
              (unsigned long long)strides[0], box_inner, box_outer);
    return false;
  }
  return true;
}

bool encode_tmap_3d(CUtensorMap *out, CUtensorMapDataType dtype, int elem_bytes,
                    const void *base, uint64_t inner, uint64_t rows, uint64_t planes,
                    uint32_t box_inner, uint32_t box_rows, CUtensorMapSwizzle swizzle) {
  if (!g_encode) {
    set_error("tensor-map encoder unavailable (hsumma_init not called?)");
    return false;
  }
  cuuint64_t dims[3] = {inner, rows, planes};
  cuuint64_t strides[2] = {inner * (uint64_t)elem_bytes, inner * rows * (uint64_t)elem_bytes};
  cuuint32_t box[3] = {box_inner, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(out, dtype, 3, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (3-D) failed (%d): %llu x %llu x %llu, box %u x %u",
              (int)r, (unsigned long long)inner, (unsigned long long)rows,
              (unsigned long long)planes, box_inner, box_rows);
    return false;
  }
  return true;
}

bool encode_tmap_kpanels(CUtensorMap *out, CUtensorMapDataType dtype, int elem_bytes,
                         const void *base, uint64_t Kp, uint64_t rows, uint64_t planes,
                         uint32_t box_rows, uint32_t kz) {
  if (!g_encode) {
    set_error("tensor-map encoder unavailable (hsumma_init not called?)");
    return false;
  }
  const uint64_t panel = 128 / (uint64_t)elem_bytes;   // elements in 128 bytes
  if (Kp % panel) {
    set_error("k-panel view needs Kp a multiple of %llu", (unsigned long long)panel);
    return false;
  }
  cuuint64_t dims[4] = {panel, rows, Kp / panel, planes};
  cuuint64_t strides[3] = {Kp * (uint64_t)elem_bytes, 128, Kp * rows * (uint64_t)elem_bytes};
  cuuint32_t box[4] = {(cuuint32_t)panel, box_rows, kz, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(out, dtype, 4, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (k panels) failed (%d): Kp %llu, rows %llu, planes %llu, "
              "box %u x %u",
              (int)r, (unsigned long long)Kp, (unsigned long long)rows,
              (unsigned long long)planes, box_rows, kz);
    return false;
  }
  return true;
}

static int launch_split_diagonals(const GridPlan &g, int kind, int S, const void *As,
                                  const void *Bs, int32_t *D, cudaStream_t s) {
  if (kind == HSUMMA_BF16_SLICES) {
    // groups of 2 x 1 and 2 x 2 processors may run on CTA pairs (clusters of
    // one or two pairs, hsumma_pair_kernel); every other shape on one CTA each
    if (g.cm == 2 && (g.cn == 1 || g.cn == 2) && g_state.bf16_pair)
      return launch_split_bf16_pair(g, S, As, Bs, D, s);
    return launch_split_bf16(g, S, As, Bs, D, s);
  }
  return launch_split_int8(g, S, As, Bs, D, s);
}

// Section III: I x J groups, I | P and J | Q; the most square in-group grid,
// ties to the smaller I.  Realised as one cluster when the group has 2..limit
// CTAs, otherwise flat.
static int resolve_groups(int P, int Q, int G, int limit, int *I, int *J, int *cm, int *cn) {
  if (P < 1 || Q < 1 || G < 1) {
    set_error("P, Q and G must be positive (got %d, %d, %d)", P, Q, G);
    return HSUMMA_ERR_ARG;
  }
  double best = -1.0;
  int bi = 0, bj = 0;
  for (int i = 1; i <= G; ++i) {
    if (G % i) continue;
    const int j = G / i;
    if (P % i || Q % j) continue;
    const double ratio = ((double)P / i) / ((double)Q / j);
    const double key = ratio >= 1.0 ? ratio : 1.0 / ratio;
    if (best < 0.0 || key < best * (1.0 - 1e-12)) {
      best = key;
      bi = i;
      bj = j;
    }
  }
  if (!bi) {
    set_error("G = %d has no factorisation I x J with I | P = %d and J | Q = %d", G, P, Q);
    return HSUMMA_ERR_ARG;
  }
  *I = bi;
  *J = bj;
  const int pi = P / bi, qj = Q / bj;
  if (pi * qj > 1 && pi * qj <= limit) {
    *cm = pi;
    *cn = qj;
  } else {
    *cm = 1;
    *cn = 1;
  }
  return HSUMMA_OK;
}

static int check_matrix_args(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda,
                             const void *B, int64_t ldb, const void *C, int64_t ldc) {
  if (M < 0 || N < 0 || K < 0) {
    set_error("negative size (M=%lld N=%lld K=%lld)", (long long)M, (long long)N,
              (long long)K);
    return HSUMMA_ERR_ARG;
  }
  if (M > (1ll << 31) || N > (1ll << 31) || K > (1ll << 31)) {
    set_error("sizes above 2^31 are not supported");
    return HSUMMA_ERR_UNSUPPORTED;
  }
  if ((M && K && lda < K) || (K && N && ldb < N) || (C && M && N && ldc < N)) {
    set_error("leading dimensions too small (lda=%lld ldb=%lld ldc=%lld)", (long long)lda,
              (long long)ldb, (long long)ldc);
    return HSUMMA_ERR_ARG;
  }
  if ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 7) {
    set_error("matrix base pointers must be 8-byte aligned");
    return HSUMMA_ERR_ARG;
  }
  if ((M && K && !A) || (K && N && !B)) {
    set_error("null matrix pointer");
    return HSUMMA_ERR_ARG;
  }
  return HSUMMA_OK;
}

// The Tensor Memory Accelerator needs 16-byte aligned bases and row strides.
static bool tma_ready(const void *p, int64_t ld) {
  return (((uintptr_t)p) & 15) == 0 && (ld & 1) == 0;
}

// kernel launches issued on the product path since the library was loaded
static std::atomic<unsigned long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n); }

}  // namespace hs

using namespace hs;

extern "C" {

int hsumma_init(int device) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_init && g_state.device == device) return HSUMMA_OK;
  if (g_init) {
    set_error("already initialised on device %d", g_state.device);
    return HSUMMA_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3) {
    set_error("device %d is sm_%d%d; the library is compiled for sm_103a", device, prop.major,
              prop.minor);
    return HSUMMA_ERR_UNSUPPORTED;
  }
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                       cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    set_error("cuTensorMapEncodeTiled entry point not found");
    return HSUMMA_ERR_CUDA;
  }
  g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  g_state = DeviceState();
  g_state.device = device;
  g_state.sm_count = prop.multiProcessorCount;
  e = cudaMalloc(&g_state.d_counters, 8 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(counters)");
  e = cudaMalloc(&g_state.d_status, 4 * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
  cudaMemset(g_state.d_counters, 0, 8 * sizeof(unsigned long long));
  cudaMemset(g_state.d_status, 0, 4 * sizeof(int));
  int lim = 16, l2 = 16;
  int st = fp64_cluster_limit(&lim);
  if (st != HSUMMA_OK) return st;
  st = bf16_cluster_limit(&l2);
  if (st != HSUMMA_OK) return st;
  if (l2 < lim) lim = l2;
  st = int8_cluster_limit(&l2);
  if (st != HSUMMA_OK) return st;
  if (l2 < lim) lim = l2;
  g_state.cluster_limit = lim;
  g_state.bf16_pair = true;   // CTA pairs for 2 x 1 groups (measured faster)
  // persistent pair clusters, split per diagonal by the library's rule: at
  // 16384^3, S = 5, B = 512 the product stage took 73.0 ms against 74.6-75.1 ms
  // with one cluster per tile and the launch rule alone (same box, interleaved)
  g_state.pair_launch = HSUMMA_PAIR_LAUNCH_AUTO | HSUMMA_PAIR_PERSISTENT;
  if (g_state.cluster_limit > 16) g_state.cluster_limit = 16;
  if (g_state.cluster_limit < 1) g_state.cluster_limit = 1;
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  g_init = true;
  return HSUMMA_OK;
}

void hsumma_finalize(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  forget_noalloc_scratch();
  if (!g_init) return;
  cudaDeviceSynchronize();
  cudaFree(g_state.d_counters);
  cudaFree(g_state.d_status);
  if (g_state.workspace) cudaFree(g_state.workspace);
  if (g_state.host_staging) cudaFree(g_state.host_staging);
  if (g_state.tune_buf) cudaFree(g_state.tune_buf);
  if (g_state.copy_in) cudaStreamDestroy(g_state.copy_in);
  if (g_state.copy_out) cudaStreamDestroy(g_state.copy_out);
  for (auto &x : g_state.pipe_ev)
    if (x) cudaEventDestroy(x);
  for (auto &x : g_state.pipe_tev)
    if (x) cudaEventDestroy(x);
  {
    std::lock_guard<std::mutex> lock(g_stage_mu);
    for (auto &ev : g_stage_ev)
      for (auto &e : ev) cudaEventDestroy(e);
    g_stage_ev.clear();
    g_stage_used = 0;
    g_stage_on = false;
  }
  forget_choices();
  forget_model_range();
  g_state = DeviceState();
  g_init = false;
}

const char *hsumma_last_error(void) { return g_err; }

int hsumma_group_shape(int P, int Q, int G, int *I, int *J, int *cluster_m, int *cluster_n) {
  if (!I || !J || !cluster_m || !cluster_n) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  const int limit = g_init ? g_state.cluster_limit : 16;
  return resolve_groups(P, Q, G, limit, I, J, cluster_m, cluster_n);
}

unsigned long long hsumma_launches(void) { return g_launches.load(); }

static int split_kind_and_S(int mode, int *kind, int *S) {
  *kind = mode & 0xff;
  *S = (mode >> 8) & 0xff;
  if (mode & ~(0xffff | HSUMMA_LAYOUT_CYCLIC)) {
    set_error("unknown mode bits %#x", mode);
    return HSUMMA_ERR_ARG;
  }
  if (*kind == HSUMMA_FP64) return HSUMMA_OK;
  if (*kind == HSUMMA_INT8_SLICES) {
    if (*S < 1 || *S > 8) {
      set_error("INT8 slices: S must be in 1..8 (got %d)", *S);
      return HSUMMA_ERR_ARG;
    }
    return HSUMMA_OK;
  }
  if (*kind == HSUMMA_BF16_SLICES) {
    if (*S < 1 || *S > 7) {
      set_error("BF16 slices: S must be in 1..7 (got %d)", *S);
      return HSUMMA_ERR_ARG;
    }
    return HSUMMA_OK;
  }
  set_error("unknown mode kind %d", *kind);
  return HSUMMA_ERR_ARG;
}

// Split-path workspace: e (M int32), f (N int32), A slices S x M x Kp,
// B slices S x N x Kp (1 or 2 bytes), exact diagonal sums S x nseg x M x N int32.
static size_t split_ws_bytes(int64_t M, int64_t N, int64_t K, int kind, int S) {
  const int64_t Kp = ceil_div(K, 64) * 64;
  const size_t eb = kind == HSUMMA_INT8_SLICES ? 1 : 2;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  return al(M * 4) + al(N * 4) + al(S * M * Kp * eb) + al(S * N * Kp * eb) +
         al((size_t)S * split_planes(K, S, kind) * M * N * 4);
}

int hsumma_workspace_size(int64_t M, int64_t N, int64_t K, int mode, size_t *bytes) {
  if (!bytes) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  int kind, S;
  int st = split_kind_and_S(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  if (M < 0 || N < 0 || K < 0) {
    set_error("negative size");
    return HSUMMA_ERR_ARG;
  }
  *bytes = kind == HSUMMA_FP64 ? 0 : split_ws_bytes(M, N, K, kind, S);
  return HSUMMA_OK;
}

static int ensure_workspace(size_t bytes) {
  if (g_state.workspace_bytes >= bytes) return HSUMMA_OK;
  if (g_state.workspace) {
    cudaDeviceSynchronize();
    cudaFree(g_state.workspace);
    g_state.workspace = nullptr;
    g_state.workspace_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&g_state.workspace, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
  g_state.workspace_bytes = bytes;
  return HSUMMA_OK;
}

static int make_plan(int64_t M, int64_t N, int64_t K, int P, int Q, int G, int b, int Bo,
                     int kind, bool cyc, GridPlan *g) {
  if (P > 65535 || Q > 65535) {
    set_error("P and Q must be at most 65535");
    return HSUMMA_ERR_ARG;
  }
  int I, J, cm, cn;
  int st = resolve_groups(P, Q, G, g_state.cluster_limit, &I, &J, &cm, &cn);
  if (st != HSUMMA_OK) return st;
  const int bmul = kind == HSUMMA_FP64 ? 16 : 64;
  if (b < bmul || b > 256 || b % bmul) {
    set_error("inner block b = %d must be a multiple of %d in %d..256", b, bmul, bmul);
    return HSUMMA_ERR_ARG;
  }
  if (Bo < b || Bo % b) {
    set_error("outer block B = %d must be a multiple of b = %d (b <= B)", Bo, b);
    return HSUMMA_ERR_ARG;
  }
  g->M = M;
  g->N = N;
  g->K = K;
  g->P = P;
  g->Q = Q;
  g->G = G;
  g->I = I;
  g->J = J;
  g->cm = cm;
  g->cn = cn;
  g->Mt = ceil_div(M, P);
  // block width rounded up so that every block starts at a column whose byte
  // offset the Tensor Memory Accelerator accepts (binary64: even columns) and
  // the split path's vector stores stay aligned (multiples of 8); the number of
  // sub-tiles per block is unchanged (tile widths are multiples of 8)
  const int64_t nal = kind == HSUMMA_FP64 ? 2 : 8;
  g->Nt = ceil_div(ceil_div(N, Q), nal) * nal;
  g->Kq = K > 0 ? ceil_div(K, Q) : 1;
  g->Kp = K > 0 ? ceil_div(K, P) : 1;
  g->nsub_m = 0;
  g->nsub_n = 0;
  g->b = b;
  g->Bo = Bo;
  g->cyc = cyc;
  if (g->Kq < 1) g->Kq = 1;
  if (g->Kp < 1) g->Kp = 1;
  return HSUMMA_OK;
}

int hsumma_gemm(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                const double *B, int64_t ldb, double *C, int64_t ldc, int P, int Q, int G,
                int b, int Bouter, int mode, void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  int st = check_matrix_args(M, N, K, A, lda, B, ldb, C, ldc);
  if (st != HSUMMA_OK) return st;
  int kind, S;
  st = split_kind_and_S(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (P == 0 && Q == 0 && G == 0 && b == 0 && Bouter == 0) {
    // automatic configuration: cached, else the loaded cost model's pick, else
    // the fastest candidate timed on these operands
    int cfg[5], how;
    st = hsumma_choose(M, N, K, A, lda, B, ldb, C, ldc, mode, HSUMMA_CHOOSE_AUTO, cfg, &how,
                       stream);
    if (st != HSUMMA_OK) return st;
    return hsumma_gemm(M, N, K, A, lda, B, ldb, C, ldc, cfg[0], cfg[1], cfg[2], cfg[3], cfg[4],
                       mode, stream);
  }
  GridPlan g;
  st = make_plan(M, N, K, P, Q, G, b, Bouter, kind, (mode & HSUMMA_LAYOUT_CYCLIC) != 0, &g);
  if (st != HSUMMA_OK) return st;
  cudaError_t e = cudaMemsetAsync(g_state.d_counters, 0, 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
  if (M == 0 || N == 0) return HSUMMA_OK;
  if (K == 0) {
    e = cudaMemset2DAsync(C, ldc * 8, 0, N * 8, M, s);
    return e == cudaSuccess ? HSUMMA_OK : cuda_fail(e, "cudaMemset2DAsync");
  }
  if (kind == HSUMMA_FP64) {
    // operands the Tensor Memory Accelerator cannot address directly (odd
    // leading dimension, base not 16-byte aligned) are copied into library
    // workspace with even row strides first
    const bool ra = !tma_ready(A, lda), rb = !tma_ready(B, ldb);
    if (ra || rb) {
      const int64_t la = (K + 1) & ~int64_t(1), lb = (N + 1) & ~int64_t(1);
      const size_t ba = ra ? ((size_t)M * la * 8 + 255) & ~size_t(255) : 0;
      const size_t bb = rb ? (size_t)K * lb * 8 : 0;
      st = ensure_workspace(ba + bb);
      if (st != HSUMMA_OK) return st;
      uint8_t *ws = reinterpret_cast<uint8_t *>(g_state.workspace);
      if (ra) {
        double *a2 = reinterpret_cast<double *>(ws);
        e = cudaMemcpy2DAsync(a2, la * 8, A, lda * 8, K * 8, M, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "repack A");
        A = a2;
        lda = la;
      }
      if (rb) {
        double *b2 = reinterpret_cast<double *>(ws + ba);
        e = cudaMemcpy2DAsync(b2, lb * 8, B, ldb * 8, N * 8, K, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "repack B");
        B = b2;
        ldb = lb;
      }
    }
    cudaEvent_t *ev = stage_slot();
    if (ev)
      for (int i = 0; i < 3; ++i) cudaEventRecord(ev[i], s);
    st = launch_fp64_hsumma(g, A, lda, B, ldb, C, ldc, s);
    if (ev)
      for (int i = 3; i < 5; ++i) cudaEventRecord(ev[i], s);
    return st;
  }

  // split path: exponents, slices, exact diagonal sums, recombination
  // exactness of the recombination: a diagonal's planes sum to at most
  // S K 2^(2w-2) in magnitude, which must fit 63 bits
  if ((double)S * (double)K * std::ldexp(1.0, 2 * slice_width(kind, S) - 2) >= 9.0e18) {
    set_error("K = %lld too large for exact slice sums with S = %d", (long long)K, S);
    return HSUMMA_ERR_UNSUPPORTED;
  }
  const size_t need = split_ws_bytes(M, N, K, kind, S);
  st = ensure_workspace(need);
  if (st != HSUMMA_OK) return st;
  const int64_t Kp = ceil_div(K, 64) * 64;
  const size_t eb = kind == HSUMMA_INT8_SLICES ? 1 : 2;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  uint8_t *ws = reinterpret_cast<uint8_t *>(g_state.workspace);
  int32_t *e_rows = reinterpret_cast<int32_t *>(ws);
  ws += al(M * 4);
  int32_t *f_cols = reinterpret_cast<int32_t *>(ws);
  ws += al(N * 4);
  void *As = ws;
  ws += al(S * M * Kp * eb);
  void *Bs = ws;
  ws += al(S * N * Kp * eb);
  int32_t *D = reinterpret_cast<int32_t *>(ws);
  cudaEvent_t *ev = stage_slot();
  if (ev) cudaEventRecord(ev[0], s);
  st = launch_split_exponents(M, N, K, A, lda, B, ldb, e_rows, f_cols, s);
  if (st != HSUMMA_OK) return st;
  if (ev) cudaEventRecord(ev[1], s);
  st = launch_split_slices(M, N, K, A, lda, B, ldb, e_rows, f_cols, kind, S, As, Bs, s);
  if (st != HSUMMA_OK) return st;
  if (ev) cudaEventRecord(ev[2], s);
  st = launch_split_diagonals(g, kind, S, As, Bs, D, s);
  if (st != HSUMMA_OK) return st;
  if (ev) cudaEventRecord(ev[3], s);
  st = launch_split_recombine(M, N, K, kind, S, D, e_rows, f_cols, C, ldc, s);
  if (ev) cudaEventRecord(ev[4], s);
  return st;
}

// Row blocks of the pipelined host-buffer product: R blocks of P/R processor
// rows each (R | P and R | I, so that every block keeps the product's blocks,
// sub-tiles and in-group grid; in the block-cyclic layout each block's tiles
// are dealt over its own P/R processor rows), at least 512 rows each, none
// empty; 1 if no R in {4, 3, 2} fits.
static int host_row_blocks(int64_t M, int P, int I, int64_t Mt) {
  for (int R : {4, 3, 2}) {
    if (R > kMaxHostBlocks || P % R || I % R) continue;
    const int64_t rows = (int64_t)(P / R) * Mt;
    if (rows < 512 || (R - 1) * rows >= M) continue;
    return R;
  }
  return 1;
}

// Column blocks likewise: 2 blocks of Q/2 processor columns (2 | Q and 2 | J)
// of at least 512 columns each, both non-empty, else 1.
static int host_col_blocks(int64_t N, int Q, int J, int64_t Nt) {
  const int C = kMaxHostColBlocks;
  if (Q % C || J % C) return 1;
  const int64_t cols = (int64_t)(Q / C) * Nt;
  if (cols < 512 || (C - 1) * cols >= N) return 1;
  return C;
}

// Row blocks in whole rounds, for products whose block products run on
// persistent CTA pairs (bf16, 2 x 1 or 2 x 2 groups, block layout): a block of
// Pr processor rows is (Pr / 2) (Qc / cn) pair tiles, swept in rounds of the
// resident clusters, so a block of t tile rows, t the least with t (Qc / cn) a
// multiple of the resident count, wastes no part of a round.  The blocks are
// the remainder of the tile rows first (small: it arrives soonest and starts
// the pipeline), then whole multiples of t, at most kMaxHostBlocks in all.
// Fills procs[] (processor rows per block) and returns the block count, or 0
// when no such split of at least two blocks exists.
static int host_row_rounds(int P, int Qc, int cn, int resident, int *procs) {
  if (resident < 1 || P % 2 || Qc % cn) return 0;
  const int u = Qc / cn, T = P / 2;          // pair tiles per tile row, tile rows
  int g = resident, h = u;
  while (h) {
    const int x = g % h;
    g = h;
    h = x;
  }
  int step = resident / g;                   // tile rows per whole number of rounds
  if (step >= T) return 0;
  int k = T / step, rem = T % step;
  const int room = kMaxHostBlocks - (rem ? 1 : 0);
  if (k > room) {
    step *= (k + room - 1) / room;
    k = T / step;
    rem = T % step;
  }
  const int nb = k + (rem ? 1 : 0);
  if (nb < 2 || nb > kMaxHostBlocks) return 0;
  int i = 0;
  if (rem) procs[i++] = 2 * rem;
  while (i < nb) procs[i++] = 2 * step;
  return nb;
}

// The pipeline's events, created on first use and kept until hsumma_finalize:
// ordering events always, timing events when `timed`.
static cudaError_t pipeline_events(bool timed) {
  cudaError_t e = cudaSuccess;
  for (auto &x : g_state.pipe_ev)
    if (!x && e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  if (timed)
    for (auto &x : g_state.pipe_tev)
      if (!x && e == cudaSuccess) e = cudaEventCreate(&x);
  return e;
}

// hsumma_gemm_host pipelined by blocks: C_rc = A_r B_c for the R row blocks of
// A and C and the Cb column blocks of B and C.  The copy-in stream brings B_0,
// A_0, then the other column blocks of B, then the other row blocks of A; the
// caller's stream, for the split path, scans and slices each column block of
// B once when it has arrived (before it waits for the row block of A it meets
// first) and each row block of A before its first product, and runs the products row block by row block (C_00, C_01, C_10, ...),
// each after the copies it needs; each finished block of C goes back on the
// copy-out stream while the next one computes.  The first product thus waits
// only for A_0 and B_0.  Every element is computed as in the unblocked product
// (row exponents are per row of A and column exponents per column of B, each
// over all of K), so the result is the same bit for bit.  With stage timing
// on, timing events bracket every phase (the timeline of hsumma_host_timeline).
static int gemm_host_pipelined(int64_t M, int64_t N, int64_t K, const double *hA, int64_t lda,
                               const double *hB, int64_t ldb, double *hC, int64_t ldc,
                               const GridPlan &full, int R, const int *procs, int Cb, int kind,
                               int S, double *dA, double *dB, double *dC, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!g_state.copy_in) e = cudaStreamCreateWithFlags(&g_state.copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !g_state.copy_out)
    e = cudaStreamCreateWithFlags(&g_state.copy_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate(copy streams)");
  bool timed;
  {
    std::lock_guard<std::mutex> lock(g_stage_mu);
    timed = g_stage_on;
  }
  e = pipeline_events(timed);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate(pipeline)");
  cudaStream_t ci = g_state.copy_in, co = g_state.copy_out;
  // row block r: processor rows procs[r], matrix rows [row0[r], row0[r] + row_count(r))
  int64_t row0[kMaxHostBlocks + 1];
  row0[0] = 0;
  for (int r = 0; r < R; ++r) row0[r + 1] = row0[r] + (int64_t)procs[r] * full.Mt;
  int64_t rows = 0;                          // the longest row block
  for (int r = 0; r < R; ++r) rows = (int64_t)procs[r] * full.Mt > rows ? (int64_t)procs[r] * full.Mt : rows;
  const int64_t cols = (int64_t)(full.Q / Cb) * full.Nt;
  auto row_count = [&](int r) {
    const int64_t end = row0[r + 1] < M ? row0[r + 1] : M;
    return end - row0[r];
  };
  auto col_count = [&](int c) { return (N - c * cols) < cols ? (N - c * cols) : cols; };
  // a small first row block: the row blocks are in whole rounds (see below)
  const bool small_first = R > 1 && procs[0] < procs[1];
  // ordering events: [0] the caller's earlier work, [1] all copied back,
  // [2 + c] B_c copied, [2 + Cb + r] A_r copied, [2 + Cb + R + (r Cb + c)] C_rc computed
  cudaEvent_t *ev = g_state.pipe_ev;
  cudaEvent_t evPrior = ev[0], evDone = ev[1];
  auto evB = [&](int c) { return ev[2 + c]; };
  auto evA = [&](int r) { return ev[2 + Cb + r]; };
  auto evC = [&](int r, int c) { return ev[2 + Cb + R + r * Cb + c]; };
  // timing events: [0] start, then (start, end) of phase i at [1 + 2 i], [2 + 2 i];
  // phases: B_c in (c < Cb), A_r in (r < R), product rc, C_rc out (r-major)
  cudaEvent_t *tev = g_state.pipe_tev;
  const int ph_b = 0, ph_a = Cb, ph_prod = Cb + R, ph_out = Cb + R + R * Cb;
  auto mark = [&](int phase, int end, cudaStream_t st) {
    return timed ? cudaEventRecord(tev[1 + 2 * phase + end], st) : cudaSuccess;
  };
  auto fail = [&](cudaError_t err, const char *what) { return cuda_fail(err, what); };

  e = cudaMemsetAsync(g_state.d_counters, 0, 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return fail(e, "cudaMemsetAsync(counters)");
  if (timed) e = cudaEventRecord(tev[0], s);
  if (e == cudaSuccess) e = cudaEventRecord(evPrior, s);  // the caller's earlier work first
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ci, evPrior, 0);
  // copies in: B_0, A_0, B_1 .., A_1 ..
  auto copy_b = [&](int c) {
    cudaError_t x = mark(ph_b + c, 0, ci);
    if (x == cudaSuccess)
      x = cudaMemcpy2DAsync(dB + c * cols, ldb * 8, hB + c * cols, ldb * 8, col_count(c) * 8, K,
                            cudaMemcpyHostToDevice, ci);
    if (x == cudaSuccess) x = mark(ph_b + c, 1, ci);
    if (x == cudaSuccess) x = cudaEventRecord(evB(c), ci);
    return x;
  };
  auto copy_a = [&](int r) {
    const int64_t r0 = row0[r];
    cudaError_t x = mark(ph_a + r, 0, ci);
    if (x == cudaSuccess)
      x = cudaMemcpy2DAsync(dA + r0 * lda, lda * 8, hA + r0 * lda, lda * 8, K * 8, row_count(r),
                            cudaMemcpyHostToDevice, ci);
    if (x == cudaSuccess) x = mark(ph_a + r, 1, ci);
    if (x == cudaSuccess) x = cudaEventRecord(evA(r), ci);
    return x;
  };
  // arrival rank of each operand block, in the order the copies are issued
  int rank_a[kMaxHostBlocks], rank_b[kMaxHostColBlocks], nrank = 0;
  auto in_b = [&](int c) { rank_b[c] = nrank++; return copy_b(c); };
  auto in_a = [&](int r) { rank_a[r] = nrank++; return copy_a(r); };
  int order[kMaxHostBlocks * kMaxHostColBlocks], nord = 0;
  if (small_first) {
    // B_0, every row block of A, then the other column blocks of B; the
    // products sweep column block 0 down the row blocks and each further
    // column block back up and down, so the last one is a small first-row
    // block's (its block of C is the last and shortest copy out)
    if (e == cudaSuccess) e = in_b(0);
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = in_a(r);
    for (int c = 1; c < Cb && e == cudaSuccess; ++c) e = in_b(c);
    for (int c = 0; c < Cb; ++c)
      for (int i = 0; i < R; ++i) order[nord++] = (c % 2 ? R - 1 - i : i) * Cb + c;
  } else {
    // B_0, A_0, the other column blocks of B, the other row blocks of A; the
    // products in the order their operands arrive (r-major among equals)
    if (e == cudaSuccess) e = in_b(0);
    if (e == cudaSuccess) e = in_a(0);
    for (int c = 1; c < Cb && e == cudaSuccess; ++c) e = in_b(c);
    for (int r = 1; r < R && e == cudaSuccess; ++r) e = in_a(r);
    for (int r = 0; r < R; ++r)
      for (int c = 0; c < Cb; ++c) order[nord++] = r * Cb + c;
    auto ready = [&](int rc) {
      const int ra = rank_a[rc / Cb], rb = rank_b[rc % Cb];
      return ra > rb ? ra : rb;
    };
    std::stable_sort(order, order + nord, [&](int x, int y) { return ready(x) < ready(y); });
  }
  if (e != cudaSuccess) return fail(e, "copy operands in");

  // split-path workspace: e (all M), f (all N), the A slices of every row
  // block and the B slices of every column block (each sliced once, at its
  // first use), the diagonal sums of one block (the block products run one
  // after another on the caller's stream)
  int32_t *e_rows = nullptr, *f_cols = nullptr, *D = nullptr;
  uint8_t *As = nullptr, *Bs = nullptr;
  size_t as_stride = 0, bs_stride = 0;
  int st = HSUMMA_OK;
  if (kind != HSUMMA_FP64) {
    const int64_t Kp = ceil_div(K, 64) * 64;
    const size_t eb = kind == HSUMMA_INT8_SLICES ? 1 : 2;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    as_stride = al((size_t)S * rows * Kp * eb);
    bs_stride = al((size_t)S * cols * Kp * eb);
    const size_t need = al(M * 4) + al(N * 4) + R * as_stride + Cb * bs_stride +
                        al((size_t)S * split_planes(K, S, kind) * rows * cols * 4);
    st = ensure_workspace(need);
    if (st != HSUMMA_OK) return st;
    uint8_t *ws = reinterpret_cast<uint8_t *>(g_state.workspace);
    e_rows = reinterpret_cast<int32_t *>(ws);
    ws += al(M * 4);
    f_cols = reinterpret_cast<int32_t *>(ws);
    ws += al(N * 4);
    As = ws;
    ws += R * as_stride;
    Bs = ws;
    ws += Cb * bs_stride;
    D = reinterpret_cast<int32_t *>(ws);
  }
  bool b_sliced[kMaxHostColBlocks] = {}, a_sliced[kMaxHostBlocks] = {};
  const int grow = full.P / full.I;          // processor rows of a group
  for (int oi = 0; oi < nord; ++oi) {
    const int r = order[oi] / Cb, c = order[oi] % Cb;
    const int64_t r0 = row0[r], mr = row_count(r);
    const double *Ar = dA + r0 * lda;
    {
      const int64_t c0 = c * cols, nc = col_count(c);
      GridPlan g;
      st = make_plan(mr, nc, K, procs[r], full.Q / Cb, (procs[r] / grow) * (full.J / Cb),
                     full.b, full.Bo, kind, full.cyc, &g);
      if (st != HSUMMA_OK) return st;
      // this block's operands: B_c (scanned and sliced at its first use, while
      // A_r may still be arriving), then A_r
      e = cudaStreamWaitEvent(s, evB(c), 0);
      if (e == cudaSuccess) e = mark(ph_prod + r * Cb + c, 0, s);
      if (e != cudaSuccess) return fail(e, "cudaStreamWaitEvent(B block)");
      double *Crc = dC + r0 * ldc + c0;
      if (kind == HSUMMA_FP64) {
        e = cudaStreamWaitEvent(s, evA(r), 0);
        if (e != cudaSuccess) return fail(e, "cudaStreamWaitEvent(A block)");
        st = launch_fp64_hsumma(g, Ar, lda, dB + c0, ldb, Crc, ldc, s);
      } else {
        void *Bsc = Bs + c * bs_stride;
        if (!b_sliced[c]) {
          b_sliced[c] = true;
          st = launch_split_exponents(0, nc, K, nullptr, 1, dB + c0, ldb, nullptr, f_cols + c0,
                                      s);
          if (st == HSUMMA_OK)
            st = launch_split_slices(0, nc, K, nullptr, 1, dB + c0, ldb, nullptr, f_cols + c0,
                                     kind, S, nullptr, Bsc, s);
        }
        e = cudaStreamWaitEvent(s, evA(r), 0);
        if (e != cudaSuccess) return fail(e, "cudaStreamWaitEvent(A block)");
        void *Asr = As + r * as_stride;
        int32_t *er = e_rows + r0;
        if (st == HSUMMA_OK && !a_sliced[r]) {
          a_sliced[r] = true;
          st = launch_split_exponents(mr, 0, K, Ar, lda, nullptr, 1, er, nullptr, s);
          if (st == HSUMMA_OK)
            st = launch_split_slices(mr, 0, K, Ar, lda, nullptr, 1, er, nullptr, kind, S, Asr,
                                     nullptr, s);
        }
        if (st == HSUMMA_OK) st = launch_split_diagonals(g, kind, S, Asr, Bsc, D, s);
        if (st == HSUMMA_OK)
          st = launch_split_recombine(mr, nc, K, kind, S, D, er, f_cols + c0, Crc, ldc, s);
      }
      if (st != HSUMMA_OK) return st;
      e = mark(ph_prod + r * Cb + c, 1, s);
      if (e == cudaSuccess) e = cudaEventRecord(evC(r, c), s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(co, evC(r, c), 0);
      if (e == cudaSuccess) e = mark(ph_out + r * Cb + c, 0, co);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(hC + r0 * ldc + c0, ldc * 8, Crc, ldc * 8, nc * 8, mr,
                              cudaMemcpyDeviceToHost, co);
      if (e == cudaSuccess) e = mark(ph_out + r * Cb + c, 1, co);
      if (e != cudaSuccess) return fail(e, "copy a block of C out");
    }
  }
  e = cudaEventRecord(evDone, co);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, evDone, 0);
  if (e != cudaSuccess) return fail(e, "join copy streams");
  st = hsumma_sync(reinterpret_cast<void *>(s));
  {
    std::lock_guard<std::mutex> lock(g_stage_mu);
    if (timed) {
      g_state.timeline_phases = st == HSUMMA_OK ? ph_out + R * Cb : 0;
      g_state.timeline_rows = R;
      g_state.timeline_cols = Cb;
    }
    g_state.host_row_blocks = R;
    for (int r = 0; r < R; ++r) g_state.host_row0[r] = row0[r];
  }
  return st;
}

int hsumma_gemm_host(int64_t M, int64_t N, int64_t K, const double *hA, int64_t lda,
                     const double *hB, int64_t ldb, double *hC, int64_t ldc, int P, int Q,
                     int G, int b, int Bouter, int mode, void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  {
    std::lock_guard<std::mutex> lock(g_stage_mu);
    g_state.timeline_phases = 0;   // set again by a timed pipelined call
    g_state.host_row_blocks = 0;   // set again by a pipelined call
  }
  int st = check_matrix_args(M, N, K, hA, lda, hB, ldb, hC, ldc);
  if (st != HSUMMA_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t bA = al((size_t)M * lda * 8), bB = al((size_t)K * ldb * 8),
               bC = al((size_t)M * ldc * 8);
  if (g_state.host_staging_bytes < bA + bB + bC) {
    if (g_state.host_staging) {
      cudaDeviceSynchronize();
      cudaFree(g_state.host_staging);
      g_state.host_staging = nullptr;
      g_state.host_staging_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&g_state.host_staging, bA + bB + bC);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(host staging)");
    g_state.host_staging_bytes = bA + bB + bC;
  }
  uint8_t *base = reinterpret_cast<uint8_t *>(g_state.host_staging);
  double *dA = reinterpret_cast<double *>(base);
  double *dB = reinterpret_cast<double *>(base + bA);
  double *dC = reinterpret_cast<double *>(base + bA + bB);
  // pipelined by row blocks when the configuration is given and allows it
  const bool given = P || Q || G || b || Bouter;
  if (given && M > 0 && N > 0 && K > 0) {
    int kind, S;
    st = split_kind_and_S(mode, &kind, &S);
    if (st != HSUMMA_OK) return st;
    GridPlan full;
    st = make_plan(M, N, K, P, Q, G, b, Bouter, kind, (mode & HSUMMA_LAYOUT_CYCLIC) != 0,
                   &full);
    if (st != HSUMMA_OK) return st;
    const bool exact_ok = kind == HSUMMA_FP64 || (double)S * (double)K * 16384.0 < 9.0e18;
    const bool tma_ok = kind != HSUMMA_FP64 || (tma_ready(dA, lda) && tma_ready(dB, ldb) &&
                                                (lda % 2) == 0);
    int R = host_row_blocks(M, P, full.I, full.Mt);
    int Cb = host_col_blocks(N, Q, full.J, full.Nt);
    // every block must resolve to the same groups and clusters as the product:
    // a block of Pr processor rows and Q / c columns has (Pr / group rows)
    // (J / c) groups
    const int grow = P / full.I;
    auto keeps_rows = [&](int Pr, int c) {
      if (Pr % grow || full.J % c) return false;
      int I, J, cm, cn;
      return resolve_groups(Pr, Q / c, (Pr / grow) * (full.J / c), g_state.cluster_limit, &I,
                            &J, &cm, &cn) == HSUMMA_OK &&
             I == Pr / grow && J == full.J / c && cm == full.cm && cn == full.cn;
    };
    if (Cb > 1 && !keeps_rows(P / R, Cb)) Cb = 1;
    if (R > 1 && !keeps_rows(P / R, Cb)) R = 1;
    int procs[kMaxHostBlocks];
    for (int r = 0; r < R; ++r) procs[r] = P / R;
    // block products on persistent CTA pairs: row blocks in whole rounds
    const bool pairs = kind == HSUMMA_BF16_SLICES && g_state.bf16_pair && full.cm == 2 &&
                       (full.cn == 1 || full.cn == 2) && !full.cyc &&
                       (g_state.pair_launch & HSUMMA_PAIR_PERSISTENT);
    int resident = 0;
    if (pairs && exact_ok && pair_resident_clusters(full.cn, &resident) == HSUMMA_OK) {
      int pr[kMaxHostBlocks];
      const int nr = host_row_rounds(P, Q / Cb, full.cn, resident, pr);
      bool ok = nr >= 2;
      for (int r = 0; r < nr && ok; ++r) ok = keeps_rows(pr[r], Cb);
      if (ok) {
        R = nr;
        for (int r = 0; r < R; ++r) procs[r] = pr[r];
      }
    }
    if (R * Cb > 1 && exact_ok && tma_ok)
      return gemm_host_pipelined(M, N, K, hA, lda, hB, ldb, hC, ldc, full, R, procs, Cb, kind,
                                 S, dA, dB, dC, s);
  }
  cudaError_t e;
  if (M && K) {
    e = cudaMemcpy2DAsync(dA, lda * 8, hA, lda * 8, K * 8, M, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(A)");
  }
  if (K && N) {
    e = cudaMemcpy2DAsync(dB, ldb * 8, hB, ldb * 8, N * 8, K, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(B)");
  }
  st = hsumma_gemm(M, N, K, dA, lda, dB, ldb, dC, ldc, P, Q, G, b, Bouter, mode, stream);
  if (st != HSUMMA_OK) return st;
  if (M && N) {
    e = cudaMemcpy2DAsync(hC, ldc * 8, dC, ldc * 8, N * 8, M, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(C)");
  }
  return hsumma_sync(stream);
}

int hsumma_get_counters(hsumma_counters *out) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  if (!out) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  unsigned long long h[8];
  cudaError_t e = cudaMemcpy(h, g_state.d_counters, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(counters)");
  out->a_loaded = h[0];
  out->a_delivered = h[1];
  out->b_loaded = h[2];
  out->b_delivered = h[3];
  out->l2_prefetch = h[4];
  out->tma_loads = h[5];
  return HSUMMA_OK;
}

int hsumma_sync(void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "kernel execution");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  int h[4];
  e = cudaMemcpy(h, g_state.d_status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
  if (h[0] != 0) {
    cudaMemset(g_state.d_status, 0, sizeof(h));
    static const char *sites[] = {"?", "stage fill", "stage release", "accumulator fill",
                                  "accumulator drain", "non-finite input", "self-test wait"};
    set_error("device error %d at %s (block %d)", h[0],
              (h[1] >= 0 && h[1] <= 6) ? sites[h[1]] : "?", h[2]);
    return h[0];
  }
  return HSUMMA_OK;
}

int hsumma_split_exponents(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                           const double *B, int64_t ldb, int32_t *e, int32_t *f,
                           void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  int st = check_matrix_args(M, N, K, A, lda, B, ldb, nullptr, 0);
  if (st != HSUMMA_OK) return st;
  if ((M && !e) || (N && !f)) {
    set_error("null exponent pointer");
    return HSUMMA_ERR_ARG;
  }
  return launch_split_exponents(M, N, K, A, lda, B, ldb, e, f,
                                reinterpret_cast<cudaStream_t>(stream));
}

int hsumma_split_slices(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                        const double *B, int64_t ldb, const int32_t *e, const int32_t *f,
                        int kind, int S, void *As, void *Bs, void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  int st = check_matrix_args(M, N, K, A, lda, B, ldb, nullptr, 0);
  if (st != HSUMMA_OK) return st;
  int k2, s2;
  st = split_kind_and_S(HSUMMA_MODE(kind, S), &k2, &s2);
  if (st != HSUMMA_OK) return st;
  if (kind == HSUMMA_FP64) {
    set_error("slices need a split kind");
    return HSUMMA_ERR_ARG;
  }
  if ((((uintptr_t)As) | ((uintptr_t)Bs)) & 15) {
    set_error("slice buffers must be 16-byte aligned");
    return HSUMMA_ERR_ARG;
  }
  return launch_split_slices(M, N, K, A, lda, B, ldb, e, f, kind, S, As, Bs,
                             reinterpret_cast<cudaStream_t>(stream));
}

int hsumma_split_planes(int64_t K, int kind, int S) {
  if (K < 0 || S < 1 || S > 8 || (kind != HSUMMA_INT8_SLICES && kind != HSUMMA_BF16_SLICES)) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  return split_planes(K, S, kind);
}

int hsumma_split_diagonals(int64_t M, int64_t N, int64_t K, int kind, int S, const void *As,
                           const void *Bs, int32_t *D, int P, int Q, int G, int b,
                           int Bouter, void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  int k2, s2;
  int st = split_kind_and_S(HSUMMA_MODE(kind, S), &k2, &s2);
  if (st != HSUMMA_OK) return st;
  if (kind == HSUMMA_FP64) {
    set_error("diagonal sums need a split kind");
    return HSUMMA_ERR_ARG;
  }
  if (M < 0 || N < 0 || K < 0 || (M && N && !D)) {
    set_error("bad sizes or null output");
    return HSUMMA_ERR_ARG;
  }
  GridPlan g;
  st = make_plan(M, N, K, P, Q, G, b, Bouter, kind, false, &g);
  if (st != HSUMMA_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(g_state.d_counters, 0, 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
  if (M == 0 || N == 0) return HSUMMA_OK;
  return launch_split_diagonals(g, kind, S, As, Bs, D, s);
}

int hsumma_split_recombine(int64_t M, int64_t N, int64_t K, int kind, int S, const int32_t *D,
                           const int32_t *e, const int32_t *f, double *C, int64_t ldc,
                           void *stream) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  int k2, s2;
  int st = split_kind_and_S(HSUMMA_MODE(kind, S), &k2, &s2);
  if (st != HSUMMA_OK) return st;
  if (M < 0 || N < 0 || ldc < N) {
    set_error("bad sizes");
    return HSUMMA_ERR_ARG;
  }
  if (M == 0 || N == 0) return HSUMMA_OK;
  if (K == 0) {
    cudaError_t e2 = cudaMemset2DAsync(C, ldc * 8, 0, N * 8, M,
                                       reinterpret_cast<cudaStream_t>(stream));
    return e2 == cudaSuccess ? HSUMMA_OK : cuda_fail(e2, "cudaMemset2DAsync");
  }
  return launch_split_recombine(M, N, K, kind, S, D, e, f, C, ldc,
                                reinterpret_cast<cudaStream_t>(stream));
}

int hsumma_peak(int kind, int64_t work, double *rate) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  if (!rate || work <= 0) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  return run_peak(kind, work, rate);
}

int hsumma_stage_timing(int enable) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  std::lock_guard<std::mutex> lock(g_stage_mu);
  g_stage_on = enable != 0;
  if (g_stage_on) g_stage_used = 0;
  return HSUMMA_OK;
}

int hsumma_stage_times(double *ms, int *calls) {
  if (!ms || !calls) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_stage_mu);
  for (int i = 0; i < 4; ++i) ms[i] = 0.0;
  for (size_t c = 0; c < g_stage_used; ++c) {
    auto &ev = g_stage_ev[c];
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(stage)");
    for (int i = 0; i < 4; ++i) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime(stage)");
      ms[i] += t;
    }
  }
  *calls = (int)g_stage_used;
  return HSUMMA_OK;
}

int hsumma_host_timeline_blocks(int *rows, int *cols) {
  if (!rows || !cols) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_stage_mu);
  *rows = g_state.timeline_phases ? g_state.timeline_rows : 0;
  *cols = g_state.timeline_phases ? g_state.timeline_cols : 0;
  return HSUMMA_OK;
}

int hsumma_host_row_rounds(int P, int Qc, int cn, int resident, int *procs, int max,
                           int *count) {
  if (!count || (max > 0 && !procs)) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  if (P < 1 || Qc < 1 || (cn != 1 && cn != 2) || resident < 1) {
    set_error("bad arguments (P=%d Qc=%d cn=%d resident=%d)", P, Qc, cn, resident);
    return HSUMMA_ERR_ARG;
  }
  int pr[kMaxHostBlocks];
  const int n = host_row_rounds(P, Qc, cn, resident, pr);
  *count = n;
  for (int r = 0; r < n && r < max; ++r) procs[r] = pr[r];
  return HSUMMA_OK;
}

int hsumma_host_row_blocks(int64_t *row0, int max, int *count) {
  if (!count || (max > 0 && !row0)) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_stage_mu);
  *count = g_state.host_row_blocks;
  for (int r = 0; r < g_state.host_row_blocks && r < max; ++r) row0[r] = g_state.host_row0[r];
  return HSUMMA_OK;
}

int hsumma_host_timeline(double *ms, int max, int *count) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  if (!count || (max > 0 && !ms)) {
    set_error("null output pointer");
    return HSUMMA_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_stage_mu);
  const int n = g_state.timeline_phases;
  *count = n;
  for (int i = 0; i < n && 2 * i + 1 < max; ++i) {
    for (int k = 0; k < 2; ++k) {
      float t = 0.f;
      cudaError_t e = cudaEventElapsedTime(&t, g_state.pipe_tev[0],
                                           g_state.pipe_tev[1 + 2 * i + k]);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime(timeline)");
      ms[2 * i + k] = t;
    }
  }
  return HSUMMA_OK;
}

int hsumma_pair_launch(int policy) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  const int was = g_state.pair_launch;
  if (policy >= 0) {
    const int split = policy & 0xf;
    if ((policy & ~(0xf | HSUMMA_PAIR_PERSISTENT)) || split > HSUMMA_PAIR_LAUNCH_PER_DIAGONAL) {
      set_error("unknown pair launch policy %#x", policy);
      return HSUMMA_ERR_ARG;
    }
    g_state.pair_launch = policy;
  }
  return was;
}

int hsumma_pair_kernel(int enable) {
  if (!g_init) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  const int was = g_state.bf16_pair ? 1 : 0;
  if (enable >= 0) g_state.bf16_pair = enable != 0;
  return was;
}

}  // extern "C"
