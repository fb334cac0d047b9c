// Automatic configuration of hsumma_gemm: which (P, Q, G, b, B) to run a
// product with.  The paper leaves the group count to a few sampled runs
// (Section V-A-1, Section VI) and fixes b and B by hand; here a candidate set is
// enumerated per product, scored by the learned cost model when one is loaded
// (hsumma_mlp_load), and otherwise timed one by one on the caller's operands
// (exhaustive search, which is also the model's judge).  Choices are cached per
// (M, N, K, mode) for the life of the process or until a model is (un)loaded.
//
// Candidate set for a product (a design of this library, not of the paper):
//   blocks of 1 or 2 sub-tiles per direction: P = ceil(M / (f_m TM)),
//   Q = ceil(N / (f_n TN)), f_m, f_n in {1, 2}, with the kernels' sub-tiles
//   TM x TN (binary64 128 x 128, int8 128 x 128, bf16 128 x 256);
//   group counts G in {1, p/16, p/8, p/4, p/2, p} (p = PQ) that factor as
//   I | P, J | Q, one per distinct realised cluster shape (flat, or a cluster
//   of the group's CTAs);
//   bf16 with an odd P > 1: also P + 1 processor rows with the groups that
//   run on CTA pairs (2 x 1 and 2 x 2), since an odd P admits none;
//   b = the kernel's stage width (32, 128, 64): b does not change the
//   arithmetic or the schedule on this GPU, only the counters' bookkeeping;
//   B in {b, 4b, 16b} (how far ahead the owners stage outer panels in L2).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"
#include "../../include/hsumma.h"

namespace hs {
namespace {

struct Cand {
  int P, Q, G, b, Bo;
};

void path_shape(int kind, int *tm, int *tn, int *b) {
  if (kind == HSUMMA_FP64) {
    *tm = 128, *tn = 128, *b = 32;
  } else if (kind == HSUMMA_INT8_SLICES) {
    *tm = 128, *tn = 128, *b = 128;
  } else {
    *tm = 128, *tn = 256, *b = 64;
  }
}

void enumerate(int64_t M, int64_t N, int kind, std::vector<Cand> &out) {
  int tm, tn, b;
  path_shape(kind, &tm, &tn, &b);
  std::vector<std::pair<int64_t, int64_t>> grids;
  // one grid's candidates: a G per distinct realised cluster shape (only the
  // CTA-pair shapes 2 x 1 and 2 x 2 when pairs_only)
  auto add_grid = [&](int64_t P, int64_t Q, bool pairs_only) {
    if (P > 65535 || Q > 65535 || P * Q > (int64_t)1 << 30) return;
    for (auto &g : grids)
      if (g.first == P && g.second == Q) return;
    grids.emplace_back(P, Q);
    const int64_t p = P * Q;
    std::vector<std::pair<int, int>> shapes;
    for (int64_t div : {p, (int64_t)16, (int64_t)8, (int64_t)4, (int64_t)2, (int64_t)1}) {
      if (p % div) continue;
      const int G = (int)(p / div);  // p / p = 1 first, then p/16 ... p
      int I, J, cm, cn;
      if (hsumma_group_shape((int)P, (int)Q, G, &I, &J, &cm, &cn) != HSUMMA_OK) continue;
      if (pairs_only && !(cm == 2 && (cn == 1 || cn == 2))) continue;
      bool dup = false;
      for (auto &s : shapes) dup |= s.first == cm && s.second == cn;
      if (dup) continue;
      shapes.emplace_back(cm, cn);
      for (int r : {1, 4, 16}) out.push_back({(int)P, (int)Q, G, b, r * b});
    }
  };
  for (int fm = 1; fm <= 2; ++fm)
    for (int fn = 1; fn <= 2; ++fn) {
      int64_t P = ceil_div(M, (int64_t)fm * tm), Q = ceil_div(N, (int64_t)fn * tn);
      if (P < 1) P = 1;
      if (Q < 1) Q = 1;
      add_grid(P, Q, false);
      // bf16: an odd P admits no CTA pairs (two processor rows each); one more
      // processor row makes them possible at the cost of a slightly
      // shorter block (M / (P + 1) rows on a 128-row tile)
      if (kind == HSUMMA_BF16_SLICES && P > 1 && (P & 1)) add_grid(P + 1, Q, true);
    }
}

void features(int64_t M, int64_t N, int64_t K, int kind, int S, const Cand &c, float *x) {
  auto lg = [](double v) { return (float)std::log2(v < 1.0 ? 1.0 : v); };
  x[0] = lg((double)M);
  x[1] = lg((double)N);
  x[2] = lg((double)K);
  x[3] = lg(c.P);
  x[4] = lg(c.Q);
  x[5] = lg(c.G);
  x[6] = lg(c.b);
  x[7] = lg(c.Bo);
  x[8] = (float)kind;
  x[9] = kind == HSUMMA_FP64 ? 0.f : (float)S;
}

std::mutex g_mu;
std::map<std::tuple<int64_t, int64_t, int64_t, int>, Cand> g_cache;

// Section IV's cost of HSUMMA with binomial broadcast trees, read for a P x Q
// grid of thread blocks with I x J groups (in-group grid (P/I) x (Q/J)):
//   inner level: each b-wide step broadcasts an Mt x b piece of A along an
//     in-group row (tree depth log2(Q/J)) and a b x Nt piece of B along an
//     in-group column (depth log2(P/I));
//   outer level: each B-wide step broadcasts Mt x B and B x Nt among the J
//     (resp. I) groups of a row (column): depth log2 J (log2 I);
//   computation: 2 Mt Nt K multiply-adds per block;
// with K counted once per slice pair on the split paths, and every term times
// the number of waves in which the grid's blocks run on the device's SMs.  For
// P = Q, I = J the latency and bandwidth factors are the paper's
// log2(p/G) n/b + log2(G) n/B and (log2(p/G) + log2(G)) n^2 / sqrt(p).  Terms:
//   [0] computation, [1] latency (messages x depth), [2] bandwidth (words x
//   depth), [3] slicing volume (M + N) K S (split paths), [4] one per call.
constexpr int kAnalyticTerms = 5;
// candidates the verified policy times: the model's best-predicted ones.  On
// the validation products (every candidate timed) the pick's geometric-mean
// ratio to the exhaustive best is 1.0033 / 1.0024 / 1.0009 / 1.0005 with 2 / 3
// / 4 / 5 timed; four keeps nearly all of the gain for one run fewer than five.
constexpr int kVerifiedCandidates = 4;
double g_analytic[3][kAnalyticTerms];
bool g_analytic_loaded = false;
// the product features (log2 M, N, K and S) the loaded model was trained on,
// per mode kind: outside them the automatic choice verifies by timing
float g_range_lo[3][kModelFeatures], g_range_hi[3][kModelFeatures];
bool g_range_loaded = false;
constexpr int kRangeFeatures[4] = {0, 1, 2, 9};

// Whether (M, N, K, S) of this kind lies inside the trained range (true when
// no range is loaded).
bool inside_trained_range(int64_t M, int64_t N, int64_t K, int kind, int S, const Cand &c) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_range_loaded) return true;
  float x[kModelFeatures];
  features(M, N, K, kind, S, c, x);
  for (int f : kRangeFeatures)
    if (!(x[f] >= g_range_lo[kind][f] - 1e-3f && x[f] <= g_range_hi[kind][f] + 1e-3f))
      return false;
  return true;
}

void analytic_terms(int64_t M, int64_t N, int64_t K, int kind, int S, const Cand &c,
                    double *f) {
  int I = 1, J = 1, cm = 1, cn = 1;
  if (hsumma_group_shape(c.P, c.Q, c.G, &I, &J, &cm, &cn) != HSUMMA_OK) I = J = 1;
  const double P = c.P, Q = c.Q, p = P * Q;
  const int sms = state().sm_count > 0 ? state().sm_count : 152;
  const double waves = std::ceil(p / sms);
  const double Mt = std::ceil((double)M / P), Nt = std::ceil((double)N / Q);
  const double pairs = kind == HSUMMA_FP64 ? 1.0 : S * (S + 1) / 2.0;
  const double Ke = (double)K * pairs;
  auto lg = [](double x) { return x > 1.0 ? std::log2(x) : 0.0; };
  const double gi = P / I, gj = Q / J;
  f[0] = waves * 2.0 * Mt * Nt * Ke;
  f[1] = waves * (Ke / c.b * (lg(gj) + lg(gi)) + Ke / c.Bo * (lg(J) + lg(I)));
  f[2] = waves * Ke * (Mt * (lg(gj) + lg(J)) + Nt * (lg(gi) + lg(I)));
  f[3] = kind == HSUMMA_FP64 ? 0.0 : (double)(M + N) * (double)K * S;
  f[4] = 1.0;
}

int decode_mode(int mode, int *kind, int *S) {
  *kind = mode & 0xff;
  *S = (mode >> 8) & 0xff;
  if (mode & ~(0xffff | HSUMMA_LAYOUT_CYCLIC)) {
    set_error("bad mode %#x", mode);
    return HSUMMA_ERR_ARG;
  }
  if (*kind == HSUMMA_FP64) return HSUMMA_OK;
  if ((*kind == HSUMMA_INT8_SLICES && *S >= 1 && *S <= 8) ||
      (*kind == HSUMMA_BF16_SLICES && *S >= 1 && *S <= 7))
    return HSUMMA_OK;
  set_error("bad mode %#x", mode);
  return HSUMMA_ERR_ARG;
}

// Score the candidates with the loaded model on the device; *best is the index
// of the smallest predicted time; with `ranked`, also every index in order of
// predicted time (the scores read back to the host).
int pick_by_model(int64_t M, int64_t N, int64_t K, int kind, int S,
                  const std::vector<Cand> &cands, cudaStream_t s, int *best,
                  std::vector<int> *ranked = nullptr) {
  float mean[kModelFeatures], stdv[kModelFeatures];
  const float *theta = loaded_model(mean, stdv);
  if (!theta) {
    set_error("no cost model loaded (hsumma_mlp_load)");
    return HSUMMA_ERR_UNSUPPORTED;
  }
  const int n = (int)cands.size();
  std::vector<float> X((size_t)n * kModelFeatures);
  for (int i = 0; i < n; ++i) {
    float *x = &X[(size_t)i * kModelFeatures];
    features(M, N, K, kind, S, cands[i], x);
    for (int j = 0; j < kModelFeatures; ++j)
      x[j] = (x[j] - mean[j]) / (stdv[j] > 0.f ? stdv[j] : 1.f);
  }
  DeviceState &st = state();
  const size_t need = ((size_t)kModelParams + (size_t)n * (kModelFeatures + 1) + 1) * 4;
  if (st.tune_bytes < need) {
    if (st.tune_buf) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
      cudaFree(st.tune_buf);
      st.tune_buf = nullptr;
      st.tune_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&st.tune_buf, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(model scoring)");
    st.tune_bytes = need;
  }
  float *d_theta = static_cast<float *>(st.tune_buf);
  float *d_X = d_theta + kModelParams;
  float *d_pred = d_X + (size_t)n * kModelFeatures;
  int32_t *d_best = reinterpret_cast<int32_t *>(d_pred + n);
  cudaError_t e = cudaMemcpyAsync(d_theta, theta, kModelParams * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_X, X.data(), X.size() * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy model inputs");
  int rc = mlp_pick_device(n, d_theta, d_X, d_pred, d_best, s);
  if (rc != HSUMMA_OK) return rc;
  int32_t h_best = -1;
  std::vector<float> pred(ranked ? n : 0);
  e = cudaMemcpyAsync(&h_best, d_best, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ranked)
    e = cudaMemcpyAsync(pred.data(), d_pred, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "read model choice");
  if (h_best < 0 || h_best >= n) {
    set_error("model choice out of range (%d of %d)", h_best, n);
    return HSUMMA_ERR_CUDA;
  }
  *best = h_best;
  if (ranked) {
    ranked->resize(n);
    for (int i = 0; i < n; ++i) (*ranked)[i] = i;
    // ascending predicted time; ties keep the candidate order (the argmin's)
    std::stable_sort(ranked->begin(), ranked->end(),
                     [&](int a, int b) { return pred[a] < pred[b]; });
  }
  return HSUMMA_OK;
}

// Time every candidate (or those listed in `only`) once on the caller's
// operands (C is overwritten) after one untimed run; *best is the fastest that
// ran.
int pick_by_timing(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                   const double *B, int64_t ldb, double *C, int64_t ldc, int mode,
                   const std::vector<Cand> &cands, cudaStream_t s, int *best,
                   const std::vector<int> *only = nullptr) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  void *sp = reinterpret_cast<void *>(s);
  float best_ms = INFINITY;
  int bi = -1;
  int rc = HSUMMA_OK;
  std::vector<int> all;
  if (!only) {
    all.resize(cands.size());
    for (size_t i = 0; i < cands.size(); ++i) all[i] = (int)i;
    only = &all;
  }
  for (int i : *only) {   // one untimed run first
    const Cand &w = cands[i];
    if (hsumma_gemm(M, N, K, A, lda, B, ldb, C, ldc, w.P, w.Q, w.G, w.b, w.Bo, mode, sp) ==
        HSUMMA_OK)
      break;
  }
  for (int i : *only) {
    const Cand &c = cands[i];
    cudaEventRecord(e0, s);
    if (hsumma_gemm(M, N, K, A, lda, B, ldb, C, ldc, c.P, c.Q, c.G, c.b, c.Bo, mode, sp) !=
        HSUMMA_OK)
      continue;  // a candidate this device cannot launch
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaEventSynchronize");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      bi = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HSUMMA_OK) return rc;
  const int sync_rc = hsumma_sync(sp);  // device-side status of the timed runs
  if (sync_rc != HSUMMA_OK) return sync_rc;
  if (bi < 0) {
    set_error("no candidate configuration ran");
    return HSUMMA_ERR_UNSUPPORTED;
  }
  *best = bi;
  return HSUMMA_OK;
}

}  // namespace

void forget_choices() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
}

void forget_model_range() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_range_loaded = false;
}

}  // namespace hs

using namespace hs;

extern "C" {

int hsumma_candidates(int64_t M, int64_t N, int64_t K, int mode, int *cfg, int max,
                      int *count) {
  int kind, S;
  int st = decode_mode(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  if (M < 0 || N < 0 || K < 0 || !count || (max > 0 && !cfg)) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  std::vector<Cand> c;
  enumerate(M, N, kind, c);
  *count = (int)c.size();
  for (int i = 0; i < (int)c.size() && i < max; ++i) {
    cfg[5 * i + 0] = c[i].P;
    cfg[5 * i + 1] = c[i].Q;
    cfg[5 * i + 2] = c[i].G;
    cfg[5 * i + 3] = c[i].b;
    cfg[5 * i + 4] = c[i].Bo;
  }
  return HSUMMA_OK;
}

int hsumma_features(int64_t M, int64_t N, int64_t K, int mode, const int *cfg, int n,
                    float *X) {
  int kind, S;
  int st = decode_mode(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  if (n < 0 || (n > 0 && (!cfg || !X))) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const Cand c{cfg[5 * i], cfg[5 * i + 1], cfg[5 * i + 2], cfg[5 * i + 3], cfg[5 * i + 4]};
    features(M, N, K, kind, S, c, X + (size_t)i * kModelFeatures);
  }
  return HSUMMA_OK;
}

int hsumma_choose(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *C, int64_t ldc, int mode, int policy,
                  int *cfg, int *how, void *stream) {
  if (state().device < 0) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  int kind, S;
  int st = decode_mode(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  if (!cfg || !how || policy < 0 || policy > HSUMMA_CHOOSE_VERIFIED || M < 0 || N < 0 ||
      K < 0) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const auto key = std::make_tuple(M, N, K, mode);
  if (policy == HSUMMA_CHOOSE_AUTO) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      const Cand &c = it->second;
      cfg[0] = c.P, cfg[1] = c.Q, cfg[2] = c.G, cfg[3] = c.b, cfg[4] = c.Bo;
      *how = HSUMMA_CHOSEN_CACHED;
      return HSUMMA_OK;
    }
  }
  std::vector<Cand> cands;
  enumerate(M, N, kind, cands);
  if (cands.empty()) {
    set_error("no candidate configuration for %lld x %lld", (long long)M, (long long)N);
    return HSUMMA_ERR_UNSUPPORTED;
  }
  int bi = 0;
  float mean[kModelFeatures], stdv[kModelFeatures];
  const bool have_model = loaded_model(mean, stdv) != nullptr;
  if (M == 0 || N == 0 || K == 0) {
    bi = 0;  // nothing to compute: any candidate does
    *how = HSUMMA_CHOSEN_MODEL;
  } else if (policy == HSUMMA_CHOOSE_ANALYTIC) {
    if (!g_analytic_loaded) {
      set_error("no analytic model loaded (hsumma_analytic_load)");
      return HSUMMA_ERR_UNSUPPORTED;
    }
    double best_t = INFINITY;
    for (size_t i = 0; i < cands.size(); ++i) {
      double f[kAnalyticTerms], t = 0.0;
      analytic_terms(M, N, K, kind, S, cands[i], f);
      for (int k = 0; k < kAnalyticTerms; ++k) t += g_analytic[kind][k] * f[k];
      if (t < best_t) {
        best_t = t;
        bi = (int)i;
      }
    }
    *how = HSUMMA_CHOSEN_ANALYTIC;
  } else if (policy == HSUMMA_CHOOSE_VERIFIED ||
             (policy == HSUMMA_CHOOSE_AUTO && have_model &&
              !inside_trained_range(M, N, K, kind, S, cands[0]))) {
    // the model's best-predicted candidates, timed on these operands (the
    // automatic choice too, for a product outside what the model was trained on)
    std::vector<int> ranked;
    st = pick_by_model(M, N, K, kind, S, cands, s, &bi, &ranked);
    if (st != HSUMMA_OK) return st;
    const bool extrapolating = policy == HSUMMA_CHOOSE_AUTO;
    std::vector<int> timed(ranked.begin(),
                           ranked.begin() + std::min(ranked.size(), (size_t)kVerifiedCandidates));
    if (extrapolating) {
      // outside the trained range the model may misjudge which kernel family
      // (cluster shape) wins, not only the panel widths: time the
      // best-predicted candidate of every cluster shape the four leave out
      std::vector<std::pair<int, int>> seen;
      auto shape_of = [&](int i) {
        int I, J, cm = 1, cn = 1;
        if (hsumma_group_shape(cands[i].P, cands[i].Q, cands[i].G, &I, &J, &cm, &cn) !=
            HSUMMA_OK)
          cm = cn = 1;
        return std::make_pair(cm, cn);
      };
      for (int i : timed) seen.push_back(shape_of(i));
      for (size_t r = timed.size(); r < ranked.size(); ++r) {
        const auto sh = shape_of(ranked[r]);
        if (std::find(seen.begin(), seen.end(), sh) != seen.end()) continue;
        seen.push_back(sh);
        timed.push_back(ranked[r]);
      }
    }
    ranked.swap(timed);
    st = pick_by_timing(M, N, K, A, lda, B, ldb, C, ldc, mode, cands, s, &bi, &ranked);
    if (st != HSUMMA_OK) return st;
    *how = HSUMMA_CHOSEN_VERIFIED;
  } else if (policy == HSUMMA_CHOOSE_MODEL || (policy == HSUMMA_CHOOSE_AUTO && have_model)) {
    st = pick_by_model(M, N, K, kind, S, cands, s, &bi);
    if (st != HSUMMA_OK) return st;
    *how = HSUMMA_CHOSEN_MODEL;
  } else {
    st = pick_by_timing(M, N, K, A, lda, B, ldb, C, ldc, mode, cands, s, &bi);
    if (st != HSUMMA_OK) return st;
    *how = HSUMMA_CHOSEN_TIMED;
  }
  const Cand &c = cands[bi];
  cfg[0] = c.P, cfg[1] = c.Q, cfg[2] = c.G, cfg[3] = c.b, cfg[4] = c.Bo;
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache[key] = c;
  return HSUMMA_OK;
}

int hsumma_analytic_terms(int64_t M, int64_t N, int64_t K, int mode, const int *cfg, int n,
                          double *terms) {
  int kind, S;
  int st = decode_mode(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  if (n < 0 || (n > 0 && (!cfg || !terms)) || M < 0 || N < 0 || K < 0) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const Cand c{cfg[5 * i], cfg[5 * i + 1], cfg[5 * i + 2], cfg[5 * i + 3], cfg[5 * i + 4]};
    if (c.P < 1 || c.Q < 1 || c.G < 1 || c.b < 1 || c.Bo < 1) {
      set_error("bad configuration");
      return HSUMMA_ERR_ARG;
    }
    analytic_terms(M, N, K, kind, S, c, terms + (size_t)i * kAnalyticTerms);
  }
  return HSUMMA_OK;
}

int hsumma_mlp_range(const float *lo, const float *hi) {
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!lo || !hi) {
      g_range_loaded = false;
    } else {
      for (int k = 0; k < 3; ++k)
        for (int f = 0; f < kModelFeatures; ++f) {
          g_range_lo[k][f] = lo[k * kModelFeatures + f];
          g_range_hi[k][f] = hi[k * kModelFeatures + f];
        }
      g_range_loaded = true;
    }
  }
  forget_choices();
  return HSUMMA_OK;
}

int hsumma_mlp_in_range(int64_t M, int64_t N, int64_t K, int mode, int *inside) {
  int kind, S;
  int st = decode_mode(mode, &kind, &S);
  if (st != HSUMMA_OK) return st;
  if (!inside || M < 0 || N < 0 || K < 0) {
    set_error("bad arguments");
    return HSUMMA_ERR_ARG;
  }
  *inside = inside_trained_range(M, N, K, kind, S, Cand{1, 1, 1, 1, 1}) ? 1 : 0;
  return HSUMMA_OK;
}

int hsumma_analytic_load(const double *coef) {
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!coef) {
      g_analytic_loaded = false;
    } else {
      for (int k = 0; k < 3; ++k)
        for (int t = 0; t < kAnalyticTerms; ++t) g_analytic[k][t] = coef[k * kAnalyticTerms + t];
      g_analytic_loaded = true;
    }
  }
  forget_choices();
  return HSUMMA_OK;
}

}  // extern "C"
