/*
 * hsumma.h -- C ABI of the single-GPU (sm_103a) Hierarchical SUMMA library.
 *
 * The library computes C = A x B (Section II-A: the product on a
 * two-dimensional grid of p = s x t processors; Section III, Algorithm 1) on
 * one GPU.  The paper's virtual processor grid becomes a grid of P x Q thread
 * blocks, one per virtual processor; its two broadcast levels become
 *   - the outer, between-group level (Section III, Figure 3): B-wide panels of
 *     A and B staged from HBM into L2 by the owner of each outer block, and
 *   - the inner, in-group level (Figure 4): b-wide panels multicast by the
 *     Tensor Memory Accelerator to every thread block of a group, the group
 *     being one thread-block cluster;
 * and the local update c_ij += a_ik b_kj runs on the tensor cores.
 *
 * Conventions for every entry point:
 *   - matrices are row-major binary64; A is M x K with leading dimension
 *     lda >= K, B is K x N (ldb >= N), C is M x N (ldc >= N); leading
 *     dimensions are counted in elements; base pointers must be 8-byte
 *     aligned.  The Tensor Memory Accelerator needs 16-byte aligned rows: with
 *     an odd leading dimension or a base that is not 16-byte aligned, the
 *     binary64 path first copies A or B into library workspace;
 *   - pointers named d_* are device pointers owned by the caller; h_* are host
 *     pointers owned by the caller; the library never frees caller memory;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); work is
 *     enqueued asynchronously, in stream order;
 *   - every call returns an hsumma_status; nothing aborts or traps.  Errors
 *     found on the device (a bounded wait that ran out, a non-finite input of
 *     the split path) are recorded in a device word and returned by the next
 *     hsumma_sync();  hsumma_last_error() gives a message for the last failure
 *     of the calling thread.
 */
#ifndef HSUMMA_H
#define HSUMMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSUMMA_OK = 0,
  HSUMMA_ERR_ARG = -1,          /* invalid argument (message says which) */
  HSUMMA_ERR_UNSUPPORTED = -2,  /* valid but outside what the library handles */
  HSUMMA_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  HSUMMA_ERR_TIMEOUT = -4,      /* a device-side bounded wait ran out */
  HSUMMA_ERR_NOT_INIT = -5,     /* hsumma_init() has not been called */
  HSUMMA_ERR_NONFINITE = -6     /* split path given an Inf or NaN input */
} hsumma_status;

/* Arithmetic of the local update.  The mode argument of hsumma_gemm carries
 * the kind in bits 0..7 and, for the split kinds, the slice count S in bits
 * 8..15: use HSUMMA_MODE(kind, S). */
typedef enum {
  HSUMMA_FP64 = 0,        /* binary64 DGEMM update (Section II-A, Algorithm 1) */
  HSUMMA_INT8_SLICES = 1, /* S int8 slices, 7 bits each, exact int32 sums, S in 1..8 */
  HSUMMA_BF16_SLICES = 2  /* S bf16 slices, 9 bits each (8 for S = 7), exact fp32 sums,
                             S in 1..7 */
} hsumma_mode;

#define HSUMMA_MODE(kind, slices) ((int)(kind) | ((int)(slices) << 8))

/* Layout of the virtual grid, or-ed into the mode argument (bit 16; other bits
 * above 15 are rejected with HSUMMA_ERR_ARG).  Without it the grid is
 * block-checkerboard (Algorithm 1): processor (r, c) owns the C block of rows
 * [r ceil(M/P), (r+1) ceil(M/P)) and columns [c Nt, (c+1) Nt), swept in
 * sub-tiles, and outer block o of A (B) is owned by the processor column
 * (row) whose share of K holds it.  With it the grid is block-cyclic, the
 * distribution Section VI leaves to future work: the sub-tiles (128 rows;
 * 128 columns for FP64 and INT8, 256 for BF16) are dealt round robin, tile row
 * t to processor row t mod P and tile column u to processor column u mod Q,
 * and outer block o is owned by processor column o mod Q (A) and row o mod P
 * (B).  Every element is the same k-ascending sum in both layouts, so C is the
 * same bit for bit; the counters follow the layout. */
#define HSUMMA_LAYOUT_CYCLIC 0x10000

/* Panel-load counters of the last hsumma_gemm launch, in matrix elements
 * (slice elements for the split kinds, counted once per slice pair).  They
 * are the GPU counterparts of the broadcast volumes of Section IV-B: with one
 * sub-tile per thread block and the group realised as one cluster,
 *   a_loaded = M K + (J-1) M K          (owner copy + outer volume),
 *   a_delivered - a_loaded = (Q-J) M K  (inner volume saved by multicast),
 * and symmetrically for B.  l2_prefetch counts outer-panel prefetches (one per
 * processor row for A and per processor column for B, per sub-tile and outer
 * step); tma_loads counts tensor-copy instructions issued. */
typedef struct {
  uint64_t a_loaded, a_delivered, b_loaded, b_delivered, l2_prefetch, tma_loads;
} hsumma_counters;

/* Bind the library to a CUDA device: queries the SM count and the largest
 * cluster size, allocates the counters and the device error word.  Must be
 * called (once per process, or again after hsumma_finalize) before any other
 * call except hsumma_group_shape, hsumma_workspace_size and
 * hsumma_last_error.  Returns HSUMMA_ERR_UNSUPPORTED on a device that is not
 * compute capability 10.3. */
int hsumma_init(int device);

/* Free everything the library allocated.  Safe to call twice.  Also drops the
 * device addresses hsumma_mlp_backward_noalloc keeps (even without
 * hsumma_init): call it after a cudaDeviceReset. */
void hsumma_finalize(void);

/* Group resolution (Section III: the s x t grid is arranged into I x J groups
 * of (s/I) x (t/J) processors; Section IV-B uses sqrt(G) x sqrt(G)).  Writes
 * the factorisation G = I J with I | P and J | Q whose in-group grid is most
 * square (ties: smaller I), and the realised cluster shape: (P/I) x (Q/J) when
 * that many thread blocks fit one cluster of the device, else 1 x 1 (the group
 * is then served flat from L2).  Before hsumma_init a cluster limit of 16 is
 * assumed.  HSUMMA_ERR_ARG if no factorisation exists. */
int hsumma_group_shape(int P, int Q, int G, int *I, int *J, int *cluster_m,
                       int *cluster_n);

/* Device workspace the library will hold for a call with these sizes and
 * mode (slices and exact pair sums of the split path; 0 for FP64).  The
 * library allocates and grows it itself on first use. */
int hsumma_workspace_size(int64_t M, int64_t N, int64_t K, int mode,
                          size_t *bytes);

/* C = A x B by HSUMMA on a virtual P x Q grid (Algorithm 1): G groups, inner
 * block b, outer block Bouter (b <= Bouter, b | Bouter; Section III requires
 * the in-group block to be no wider than the between-group one).  Blocks are ceil(M/P) x ceil(N/Q) and the last ones may
 * be short (the paper assumes divisibility; short blocks are allowed here);
 * 1 <= P, Q <= 65535; G must factor as above; b a multiple of 16 in 16..256
 * for FP64 and of 64 in 64..256 for the split kinds; Bouter a multiple of b.
 * P = Q = G = b = Bouter = 0 asks the library to choose them
 * (the learned cost model if one is loaded, else exhaustive timing of the
 * candidate set).  C is overwritten (beta = 0).  M, N or K = 0 is allowed
 * (K = 0 writes zeros).  The split kinds (Ozaki-style error-free slicing)
 * need finite inputs and K small enough for exact integer sums. */
int hsumma_gemm(int64_t M, int64_t N, int64_t K, const double *d_A, int64_t lda,
                const double *d_B, int64_t ldb, double *d_C, int64_t ldc, int P,
                int Q, int G, int b, int Bouter, int mode, void *stream);

/* The same product from host buffers: copies A and B to library-owned device
 * buffers, runs hsumma_gemm, copies C back and synchronises the stream.
 * Pinned host memory gives full copy bandwidth; pageable memory works. */
int hsumma_gemm_host(int64_t M, int64_t N, int64_t K, const double *h_A,
                     int64_t lda, const double *h_B, int64_t ldb, double *h_C,
                     int64_t ldc, int P, int Q, int G, int b, int Bouter,
                     int mode, void *stream);

/* Counters of the last hsumma_gemm launch (call after hsumma_sync). */
int hsumma_get_counters(hsumma_counters *out);

/* Number of kernel launches the library has issued for products (exponent
 * scan, slicing, products, recombination; binary64: the product kernel) since
 * it was loaded.  Read it before and after a region to count that region's
 * launches.  Host-side count; needs no device and no hsumma_init. */
unsigned long long hsumma_launches(void);

/* Synchronise `stream` and report device-side errors recorded since the last
 * call (HSUMMA_ERR_TIMEOUT, HSUMMA_ERR_NONFINITE) or a CUDA error. */
int hsumma_sync(void *stream);

/* Message of the calling thread's last failure ("" if none). */
const char *hsumma_last_error(void);

/* ---- Split path, step by step (the steps hsumma_gemm runs for the split
 * kinds; exposed so that each step can be checked on its own) ---- */

/* Step 1, exponent scan: e[i] = ilogb(max_k |A_ik|) + 2 (0 for a zero row),
 * f[j] likewise over the columns of B, so that every scaled entry is < 1/2 in
 * magnitude.  d_e: M int32, d_f: N int32. */
int hsumma_split_exponents(int64_t M, int64_t N, int64_t K, const double *d_A,
                           int64_t lda, const double *d_B, int64_t ldb,
                           int32_t *d_e, int32_t *d_f, void *stream);

/* Step 2, slicing: digit s (s = 1..S) of every entry, t_s = rint(r 2^(w s)) -
 * 2^w rint(r 2^(w (s-1))), r = A_ik 2^-e_i (round half to even), written as
 * int8 (kind INT8, w = 7: digits in [-64, 64]) or bf16 (kind BF16, w = 9:
 * digits in [-256, 256], every one exact in bfloat16; w = 8 for S = 7, since
 * w S <= 56).  Layout: d_As is
 * S x M x Kp (row-major, Kp = K rounded up to a multiple of 64, zero padded),
 * d_Bs is S x N x Kp (B transposed: row j of slice t holds column j of B). */
int hsumma_split_slices(int64_t M, int64_t N, int64_t K, const double *d_A,
                        int64_t lda, const double *d_B, int64_t ldb,
                        const int32_t *d_e, const int32_t *d_f, int kind, int S,
                        void *d_As, void *d_Bs, void *stream);

/* Number of int32 planes per diagonal that step 3 writes for this K: a
 * diagonal's exact sum is split into segments whose partial sums stay below
 * 2^31 in magnitude (bf16: 127 x 2^(26-2w) products -- 127 x 256 for w = 9,
 * 127 x 1024 for w = 8 -- int8: 2^18).  The count
 * covers the longest diagonal, S pairs of K rounded up to a multiple of 128
 * (the product kernels' stage width); every plane of every diagonal is
 * written, zeros past a diagonal's own segments.  Returns the count (>= 1)
 * or HSUMMA_ERR_ARG. */
int hsumma_split_planes(int64_t K, int kind, int S);

/* Step 3, the kept pair products (pairs s + t <= S + 1) multiplied on the
 * tensor cores with HSUMMA's data movement (arguments P..Bouter as in
 * hsumma_gemm), summed exactly per diagonal d = s + t:
 * D_d[i][j] = sum_{s+t=d} sum_k a_s[i,k] b_t[k,j] = sum_g d_D[d-2][g][i][j]
 * over the g = 0..hsumma_split_planes(K, kind, S)-1 int32 planes of d_D
 * (layout S x planes x M x N).  d_As and d_Bs as written by step 2. */
int hsumma_split_diagonals(int64_t M, int64_t N, int64_t K, int kind, int S,
                           const void *d_As, const void *d_Bs, int32_t *d_D,
                           int P, int Q, int G, int b, int Bouter, void *stream);

/* Step 4, recombination: C_ij = RN(2^(e_i + f_j) sum_d D_d,ij 2^(-w d)), the
 * exact sum (64- or 128-bit integers) rounded once to binary64, ties to even,
 * subnormal and overflowing results included.  Only the planes of a diagonal
 * that step 3 can fill are read (the others hold zeros). */
int hsumma_split_recombine(int64_t M, int64_t N, int64_t K, int kind, int S,
                           const int32_t *d_D, const int32_t *d_e,
                           const int32_t *d_f, double *d_C, int64_t ldc,
                           void *stream);

/* ---- Learned cost model (not in the paper: the paper picks G by sampling a
 * few runs, Section V-A-1 and Section VI) ---- */

/* MLP 10 -> 64 -> 64 -> 64 -> 1 with exact GELU; parameter vector layout
 * W1[64][10] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[1][64] b4[1]
 * (9089 floats).  Forward in fp32: d_X batch x 10, d_y batch predictions;
 * d_cache (batch x 192 floats of pre-activations) may be NULL. */
int hsumma_mlp_forward(int batch, const float *d_theta, const float *d_X,
                       float *d_y, float *d_cache, void *stream);

/* Gradient of mean_i (f(x_i) - t_i)^2 with respect to the parameters (fp32),
 * and the loss: d_grad 9089 floats, d_loss 1 float.  The per-block partial
 * gradients live in a buffer of the call itself, taken from and returned to
 * the current device's stream-ordered memory pool on `stream`
 * (cudaMallocAsync / cudaFreeAsync), so calls on different devices, streams
 * or host threads do not share it. */
int hsumma_mlp_backward(int batch, const float *d_theta, const float *d_X,
                        const float *d_target, float *d_grad, float *d_loss,
                        void *stream);

/* hsumma_mlp_backward without allocation.  The paper has no counterpart: this
 * is a library facility for callers that must not allocate device memory once
 * they are running, such as a serving process that refines its cost model
 * between requests while its memory is fully planned (or held by a caching
 * allocator), or one that cannot take the device-wide synchronisation that
 * cudaMalloc and cudaFree bring while other streams are busy.
 * hsumma_mlp_backward takes a buffer of per-block partial gradients from the
 * stream-ordered pool (cudaMallocAsync) on every call; this variant keeps them
 * in one fixed array in the library's device image (about 18.6 MB, held by
 * every device that loads the library until the process exits) and calls no
 * cudaMalloc, cudaFree or allocating routine.  Arguments, layout and results
 * are those of hsumma_mlp_backward; the caller passes every input and output.
 *   batch: 1..HSUMMA_MLP_NOALLOC_MAX_BATCH; a larger batch returns
 *          HSUMMA_ERR_ARG (message in hsumma_last_error) and launches nothing.
 * The first call on each device (with that device current) looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it; make that first
 * call before any stream capture.  A cudaDeviceReset invalidates the kept
 * address: call hsumma_finalize after such a reset (it drops the kept
 * addresses, whether or not hsumma_init was called) so that the next call
 * looks them up again.  All calls share the array and it keeps the last call's
 * contents (nothing in it needs clearing, every slot read is written first in
 * the same call): calls that overlap on the GPU, on different streams or from
 * different host threads, race and give wrong gradients. */
#define HSUMMA_MLP_NOALLOC_MAX_BATCH 4096
int hsumma_mlp_backward_noalloc(int batch, const float *d_theta, const float *d_X,
                                const float *d_target, float *d_grad, float *d_loss,
                                void *stream);

/* One Adam step (fp32), step number t >= 1, on n parameters. */
int hsumma_mlp_adam(int n, float *d_theta, const float *d_grad, float *d_m,
                    float *d_v, int t, float lr, float beta1, float beta2,
                    float eps, void *stream);

/* Score candidates with the model in bf16 and return the index of the
 * smallest prediction: d_X n x 10 features (already normalised). */
int hsumma_mlp_pick(int n, const float *d_theta, const float *d_X,
                    float *d_pred, int32_t *d_best, void *stream);

/* Load a trained model into the library (host arrays: 9089 parameters, the
 * 10 feature means and 10 standard deviations) for hsumma_gemm's automatic
 * choice; NULL theta unloads it.  Either way every cached choice and the
 * trained range (hsumma_mlp_range) are dropped. */
int hsumma_mlp_load(const float *h_theta, const float *h_mean,
                    const float *h_std);

/* ---- Automatic configuration ----
 * The paper picks the group count by timing a few runs (Section V-A-1,
 * Section VI) and fixes b and B by hand.  Here the candidates for a product
 * are enumerated by the library, scored by the loaded cost model, or timed one
 * by one (exhaustive search: the fallback, and the yardstick of the model). */

/* Candidate configurations for a product: *count = their number (at most 72);
 * the first min(count, max) are written to cfg as (P, Q, G, b, Bouter)
 * quintuples.  Blocks of 1 or 2 kernel sub-tiles per direction; group counts
 * 1, p/16, p/8, p/4, p/2 and p (p = PQ), one per distinct realised cluster
 * shape; b = the kernel's stage width (32 FP64, 128 INT8, 64 BF16), which does
 * not change the schedule on this GPU; Bouter in {b, 4b, 16b}.  Host only. */
int hsumma_candidates(int64_t M, int64_t N, int64_t K, int mode, int *h_cfg,
                      int max, int *h_count);

/* The cost model's 10 input features of n configurations (h_cfg: n
 * quintuples as above), written to h_X (n x 10 floats, row-major):
 * log2 of M, N, K, P, Q, G, b, Bouter; the mode kind (0, 1, 2); S (0 for
 * FP64).  The model sees them standardised with the loaded means and
 * deviations.  Host only. */
int hsumma_features(int64_t M, int64_t N, int64_t K, int mode,
                    const int *h_cfg, int n, float *h_X);

/* Choice policies and how a choice was made. */
enum {
  HSUMMA_CHOOSE_AUTO = 0,     /* cached, else the model (verified by timing outside its
                                 trained range, hsumma_mlp_range), else timing */
  HSUMMA_CHOOSE_MODEL = 1,    /* the loaded model (HSUMMA_ERR_UNSUPPORTED if none) */
  HSUMMA_CHOOSE_TIMED = 2,    /* exhaustive timing, always */
  HSUMMA_CHOOSE_ANALYTIC = 3, /* the fitted analytic model (hsumma_analytic_load) */
  HSUMMA_CHOOSE_VERIFIED = 4  /* the model's four best-predicted candidates, timed */
};
enum {
  HSUMMA_CHOSEN_CACHED = 0,
  HSUMMA_CHOSEN_MODEL = 1,
  HSUMMA_CHOSEN_TIMED = 2,
  HSUMMA_CHOSEN_ANALYTIC = 3,
  HSUMMA_CHOSEN_VERIFIED = 4
};

/* Section IV's cost model of HSUMMA with binomial broadcast trees, read for a
 * P x Q grid of thread blocks with I x J groups (in-group grid (P/I) x (Q/J)),
 * blocks Mt x Nt = ceil(M/P) x ceil(N/Q), K counted once per slice pair on the
 * split paths (Ke = K or K S(S+1)/2) and W = ceil(PQ / SMs) waves.  Writes
 * 5 terms per configuration to h_terms (n x 5, row-major):
 *   [0] computation  W 2 Mt Nt Ke,
 *   [1] latency      W (Ke/b (log2(Q/J) + log2(P/I)) + Ke/B (log2 J + log2 I)),
 *   [2] bandwidth    W Ke (Mt (log2(Q/J) + log2 J) + Nt (log2(P/I) + log2 I)),
 *   [3] slicing      (M + N) K S on the split paths (0 for FP64),
 *   [4] 1 (per call).
 * For P = Q and I = J, [1] and [2] are the latency factor
 * log2(p/G) n/b + log2(G) n/B and the bandwidth factor
 * (log2(p/G) + log2 G) n^2/sqrt(p) of Section IV (Table I) times W.
 * The predicted time is the dot product with the coefficients (gamma, alpha,
 * beta, slicing, overhead) loaded by hsumma_analytic_load.  Host only. */
int hsumma_analytic_terms(int64_t M, int64_t N, int64_t K, int mode,
                          const int *h_cfg, int n, double *h_terms);

/* The product features the loaded model was trained on, per mode kind:
 * h_lo and h_hi hold 3 x 10 floats (kind-major, the features of
 * hsumma_features), of which log2 M, log2 N, log2 K and S are used.  A product
 * outside them for its kind (by more than 1e-3) makes the automatic choice
 * (HSUMMA_CHOOSE_AUTO) time candidates instead of taking the model's pick (the
 * model extrapolates there; hsumma_choose says which).  A kind without training samples has lo > hi.
 * NULL clears the range (the model is then used everywhere), and so do
 * hsumma_mlp_load and hsumma_finalize: load the range after its model.  Drops
 * every cached choice.  Host only. */
int hsumma_mlp_range(const float *h_lo, const float *h_hi);

/* *h_inside = 1 when the product (M, N, K, mode) lies inside the loaded
 * trained range for its kind (or no range is loaded), else 0: whether the
 * automatic choice takes the model's pick or verifies it by timing.  Host
 * only. */
int hsumma_mlp_in_range(int64_t M, int64_t N, int64_t K, int mode, int *h_inside);

/* Coefficients of the analytic model, 5 per mode kind (FP64, INT8, BF16),
 * h_coef[kind * 5 + term] (seconds per unit of each term); NULL unloads.
 * Drops every cached choice. */
int hsumma_analytic_load(const double *h_coef);

/* The configuration hsumma_gemm runs with when P = Q = G = b = Bouter = 0:
 * written to h_cfg[5] with *h_how one of HSUMMA_CHOSEN_*.  The model scores
 * every candidate on the device (bf16) and takes the smallest predicted time;
 * timing runs every candidate once on these operands, after one untimed run,
 * overwriting C, and takes the fastest that launched; the verified policy
 * times only the model's four best-predicted candidates the same way.  The
 * automatic choice, for a product outside the model's trained range, times
 * those four and the best-predicted candidate of every cluster shape
 * (hsumma_group_shape) they leave out.
 * Either way the stream is synchronised and the choice is cached per
 * (M, N, K, mode) until the next hsumma_mlp_load, hsumma_mlp_range or
 * hsumma_finalize.  Operands follow hsumma_gemm's rules (they are only read by
 * timing). */
int hsumma_choose(int64_t M, int64_t N, int64_t K, const double *d_A,
                  int64_t lda, const double *d_B, int64_t ldb, double *d_C,
                  int64_t ldc, int mode, int policy, int *h_cfg, int *h_how,
                  void *stream);

/* Kernel choice for the bf16 split path when a group is realised as a 2 x 1
 * cluster (two vertically adjacent processors, e.g. G = p/2): enable = 1 runs
 * its products on CTA pairs (tcgen05 cta_group::2: each SM holds its own A rows
 * and half of the shared B panel, and the pair MMA reads both halves -- the
 * in-group broadcast of Section III done by the tensor cores; the setting
 * after hsumma_init); 0 runs the single-CTA kernel; a negative value only
 * queries.  Returns the previous setting (0 or 1), or HSUMMA_ERR_NOT_INIT.
 * Results are identical either way. */
int hsumma_pair_kernel(int enable);

/* Launch policy of the CTA-pair kernel (hsumma_pair_kernel).  The low four
 * bits choose how the slice pairs are split over launches:
 *   HSUMMA_PAIR_LAUNCH_AUTO          the library's rule: one launch per
 *                                    diagonal for long products of many
 *                                    rounds of tiles, else one launch;
 *   HSUMMA_PAIR_LAUNCH_ONE           one launch for all S (S + 1) / 2 pairs;
 *   HSUMMA_PAIR_LAUNCH_PER_DIAGONAL  one launch per diagonal d = s + t;
 * or-ing HSUMMA_PAIR_PERSISTENT launches one cluster per resident cluster
 * slot of the device, each sweeping the group tiles cid, cid + ncl, ...,
 * instead of one cluster per group tile; a launch for all diagonals then
 * cuts the tiles past its last whole round into one item per diagonal and
 * deals them to the least-loaded clusters.  After hsumma_init the policy is
 * HSUMMA_PAIR_LAUNCH_AUTO | HSUMMA_PAIR_PERSISTENT.  A negative value only
 * queries.
 * Returns the previous policy, HSUMMA_ERR_ARG for an unknown one, or
 * HSUMMA_ERR_NOT_INIT.  Results are identical under every policy. */
enum {
  HSUMMA_PAIR_LAUNCH_AUTO = 0,
  HSUMMA_PAIR_LAUNCH_ONE = 1,
  HSUMMA_PAIR_LAUNCH_PER_DIAGONAL = 2
};
#define HSUMMA_PAIR_PERSISTENT 0x10
int hsumma_pair_launch(int policy);

/* Self-test of the failure handling (the paper has no counterpart): launches
 * one block that waits on a shared-memory barrier nothing arrives on, gives up
 * after limit_ns (0 .. 1e9) of device time, and records HSUMMA_ERR_TIMEOUT in
 * the device status word exactly as a GEMM kernel whose wait ran out would;
 * the next hsumma_sync on the stream returns HSUMMA_ERR_TIMEOUT ("self-test
 * wait") and clears the word.  Nothing faults or hangs. */
int hsumma_selftest_timeout(long long limit_ns, void *stream);

/* ---- Stage timing ----
 * Per-kernel device time of hsumma_gemm on the caller's stream, for measuring
 * the path while it runs.  hsumma_stage_timing(1) clears the record and makes
 * every following hsumma_gemm call record five CUDA events around its stages
 * (on the call's stream); hsumma_stage_timing(0) stops recording.
 * hsumma_stage_times waits for the recorded events and writes the summed
 * milliseconds of the four stages over the recorded calls to h_ms[4] (split
 * path: exponent scan, slicing, diagonal products, recombination; binary64:
 * 0, 0, the product kernel, 0) and their number to *h_calls.  An event pair is
 * read only once its call has finished; a call that failed part-way leaves
 * unrecorded events and makes hsumma_stage_times fail. */
int hsumma_stage_timing(int enable);
int hsumma_stage_times(double *h_ms, int *h_calls);

/* hsumma_gemm_host runs a product of at least two blocks as a pipeline: C is
 * cut into R row blocks (R in {4, 3, 2}, R | P, R | I; blocks of other sizes
 * for products on persistent CTA pairs, see hsumma_host_row_blocks) and Cb
 * column blocks (Cb in {2, 1}, Cb | Q, Cb | J), each block keeping the
 * product's groups; B_0 and A_0 are copied in first; each block's work starts
 * once its B_c is on the device (the split path scans and slices B_c there,
 * at its first use) and its product once A_r is too, while the rest copy in
 * and the finished blocks of C copy out.
 * Timeline of the last hsumma_gemm_host call, when that call ran with stage
 * timing on and was pipelined (otherwise *h_count = 0): *h_count phases, in
 * this order: the copies of B_c in (c < Cb), the copies of A_r in (r < R),
 * the block products (indexed r-major: C_00, C_01, C_10, ...; each from the moment
 * its B_c is on the device, so the first includes the wait for A_0), the
 * copies of the blocks of C out (same order).  For phase i, h_ms[2 i] and
 * h_ms[2 i + 1] are
 * its start and end in milliseconds after the call's first event (CUDA events
 * on the stream that ran the phase); at most max values are written (at most
 * 22 phases).  hsumma_host_timeline_blocks gives R and Cb of that call (0 and
 * 0 when there is no timeline). */
int hsumma_host_timeline(double *h_ms, int max, int *h_count);
int hsumma_host_timeline_blocks(int *rows, int *cols);

/* The row blocks of the last hsumma_gemm_host call (timed or not): their count
 * in *h_count (0 if that call was not pipelined) and the first row of each in
 * h_row0[0 .. min(count, max) - 1].  Uniform blocks of P/R processor rows,
 * except for bf16 products whose blocks run on persistent CTA pairs (2 x 1 or
 * 2 x 2 groups, block layout): there every block after the first spans a
 * whole number of rounds of the resident pair clusters, and the first block
 * takes the remaining rows (it is copied in and computed first; every row
 * block of A is then copied before the other column blocks of B, and the
 * block products sweep column block 0 down the row blocks and the next one
 * back up, so that the last block of C copied out is a small one).  Returns
 * HSUMMA_ERR_ARG on a null pointer. */
int hsumma_host_row_blocks(int64_t *h_row0, int max, int *h_count);

/* The round-aligned row blocks that rule gives for a grid of P processor rows
 * (pairs of rows: P even), Qc processor columns per column block, CTA pairs
 * of cn in {1, 2} columns and `resident` clusters: t = the least number of
 * tile rows (pairs of processor rows) whose (Qc / cn) t pair tiles are a
 * multiple of `resident`; blocks of t tile rows (of a multiple of t when
 * more than 4 blocks would result), the remainder first.  Writes the
 * processor rows of each block to procs[0 .. min(count, max) - 1] and their
 * count (2 to 4) to *h_count, or 0 when no split of at least two blocks
 * exists (P odd, t >= P / 2).  Host arithmetic only.  Returns HSUMMA_ERR_ARG
 * on a null pointer or an argument out of range. */
int hsumma_host_row_rounds(int P, int Qc, int cn, int resident, int *procs, int max,
                           int *h_count);

/* ---- Peak microbenchmarks (roofline denominators) ---- */

typedef enum {
  HSUMMA_PEAK_DFMA = 0,      /* binary64 FMA on the CUDA cores */
  HSUMMA_PEAK_DMMA = 1,      /* binary64 mma.sync m16n8k4 */
  HSUMMA_PEAK_IMMA = 2,      /* int8 mma.sync m16n8k32, int32 accumulate */
  HSUMMA_PEAK_HMMA_BF16 = 3, /* bf16 mma.sync m16n8k16, fp32 accumulate */
  HSUMMA_PEAK_TC05_BF16 = 4, /* bf16 tcgen05.mma 128x256x16, fp32 in TMEM */
  HSUMMA_PEAK_COPY = 5,      /* device memory copy (bytes read + written) */
  HSUMMA_PEAK_TC05_BF16_PAIR = 6 /* bf16 tcgen05.mma cta_group::2 256x256x16 */
} hsumma_peak_kind;

/* Run one microbenchmark on every SM and return the rate: flops/s (2 per
 * multiply-add) or bytes/s for the copy.  `work` scales the run length. */
int hsumma_peak(int kind, int64_t work, double *rate);

#ifdef __cplusplus
}
#endif

#endif /* HSUMMA_H */
