// Learned cost model: a 10 -> 64 -> 64 -> 64 -> 1 MLP with exact GELU,
// trained in fp32 (forward, backpropagation, Adam) and run in bf16 to score the
// candidate configurations of a product.  Not in the paper, which picks the
// group count by sampling a few runs (Section V-A-1, Section VI); this model
// proposes (P, Q, G, b, B) from the features of a shape instead.
//
// Parameter vector layout (row-major W[out][in]):
//   W1[64][10] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[1][64] b4[1]
// Every kernel keeps the weights in shared memory (36 KB) and gives one sample
// to each warp (lane j computes neurons j and j + 32); each block accumulates
// its samples' gradient in shared memory, and the block partials are summed in
// block order by a second kernel.
#include <cuda_bf16.h>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int NIN = 10, NH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH,
              OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NH, NPARAM = OFF_B4 + 1;
static_assert(NPARAM == 9089, "parameter count");
constexpr int WARPS = 8;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// h_out[j] = W[j][:] . h_in + b[j] for this lane's two neurons (j, j + 32);
// h_in lives in shared memory, one row per warp.
template <int NI>
__device__ __forceinline__ void dense2(const float *W, const float *b, const float *h_in,
                                       int lane, float &z0, float &z1) {
  float a0 = b[lane], a1 = b[lane + 32];
#pragma unroll 8
  for (int i = 0; i < NI; ++i) {
    const float x = h_in[i];
    a0 = fmaf(W[lane * NI + i], x, a0);
    a1 = fmaf(W[(lane + 32) * NI + i], x, a1);
  }
  z0 = a0;
  z1 = a1;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(WARPS * 32) mlp_forward_kernel(int batch, const float *theta,
                                                                  const float *X, float *y,
                                                                  float *cache) {
  __shared__ float w[NPARAM];
  __shared__ float h[WARPS][3][NH];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = theta[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int smp = blockIdx.x * WARPS + warp; smp < batch; smp += gridDim.x * WARPS) {
    float *hin = h[warp][0];
    if (lane < NIN) hin[lane] = X[(int64_t)smp * NIN + lane];
    __syncwarp();
    float z0, z1;
    dense2<NIN>(w + OFF_W1, w + OFF_B1, hin, lane, z0, z1);
    if (cache) {
      cache[(int64_t)smp * 192 + lane] = z0;
      cache[(int64_t)smp * 192 + lane + 32] = z1;
    }
    h[warp][1][lane] = gelu(z0);
    h[warp][1][lane + 32] = gelu(z1);
    __syncwarp();
    dense2<NH>(w + OFF_W2, w + OFF_B2, h[warp][1], lane, z0, z1);
    if (cache) {
      cache[(int64_t)smp * 192 + 64 + lane] = z0;
      cache[(int64_t)smp * 192 + 96 + lane] = z1;
    }
    h[warp][2][lane] = gelu(z0);
    h[warp][2][lane + 32] = gelu(z1);
    __syncwarp();
    dense2<NH>(w + OFF_W3, w + OFF_B3, h[warp][2], lane, z0, z1);
    if (cache) {
      cache[(int64_t)smp * 192 + 128 + lane] = z0;
      cache[(int64_t)smp * 192 + 160 + lane] = z1;
    }
    const float out = warp_sum(w[OFF_W4 + lane] * gelu(z0) + w[OFF_W4 + lane + 32] * gelu(z1));
    if (lane == 0) y[smp] = out + w[OFF_B4];
    __syncwarp();
  }
}

// Per-block partial gradient of mean_i (f(x_i) - t_i)^2 (and partial loss).
__global__ void __launch_bounds__(WARPS * 32)
    mlp_backward_kernel(int batch, const float *theta, const float *X, const float *target,
                        float *partial, float *partial_loss) {
  extern __shared__ float dyn[];
  float *w = dyn, *gw = dyn + NPARAM;
  __shared__ float h0[WARPS][NIN];
  __shared__ float h1[WARPS][NH], h2[WARPS][NH], h3[WARPS][NH];
  __shared__ float g3[WARPS][NH], g2[WARPS][NH];
  __shared__ float lossw[WARPS];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    w[i] = theta[i];
    gw[i] = 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float loss = 0.f;
  for (int smp = blockIdx.x * WARPS + warp; smp < batch; smp += gridDim.x * WARPS) {
    if (lane < NIN) h0[warp][lane] = X[(int64_t)smp * NIN + lane];
    __syncwarp();
    float z1a, z1b, z2a, z2b, z3a, z3b;
    dense2<NIN>(w + OFF_W1, w + OFF_B1, h0[warp], lane, z1a, z1b);
    h1[warp][lane] = gelu(z1a);
    h1[warp][lane + 32] = gelu(z1b);
    __syncwarp();
    dense2<NH>(w + OFF_W2, w + OFF_B2, h1[warp], lane, z2a, z2b);
    h2[warp][lane] = gelu(z2a);
    h2[warp][lane + 32] = gelu(z2b);
    __syncwarp();
    dense2<NH>(w + OFF_W3, w + OFF_B3, h2[warp], lane, z3a, z3b);
    h3[warp][lane] = gelu(z3a);
    h3[warp][lane + 32] = gelu(z3b);
    __syncwarp();
    const float out =
        warp_sum(w[OFF_W4 + lane] * h3[warp][lane] + w[OFF_W4 + lane + 32] * h3[warp][lane + 32]) +
        w[OFF_B4];
    const float diff = out - target[smp];
    loss += diff * diff;
    const float gy = 2.0f * diff / (float)batch;
    // layer 4
    atomicAdd(&gw[OFF_W4 + lane], gy * h3[warp][lane]);
    atomicAdd(&gw[OFF_W4 + lane + 32], gy * h3[warp][lane + 32]);
    if (lane == 0) atomicAdd(&gw[OFF_B4], gy);
    // layer 3: dz3 = W4 gy * gelu'(z3)
    const float d3a = w[OFF_W4 + lane] * gy * gelu_grad(z3a);
    const float d3b = w[OFF_W4 + lane + 32] * gy * gelu_grad(z3b);
    g3[warp][lane] = d3a;
    g3[warp][lane + 32] = d3b;
    __syncwarp();
    for (int i = 0; i < NH; ++i) {
      atomicAdd(&gw[OFF_W3 + lane * NH + i], d3a * h2[warp][i]);
      atomicAdd(&gw[OFF_W3 + (lane + 32) * NH + i], d3b * h2[warp][i]);
    }
    atomicAdd(&gw[OFF_B3 + lane], d3a);
    atomicAdd(&gw[OFF_B3 + lane + 32], d3b);
    // layer 2: dh2 = W3^T dz3
    float s2a = 0.f, s2b = 0.f;
    for (int o = 0; o < NH; ++o) {
      s2a = fmaf(w[OFF_W3 + o * NH + lane], g3[warp][o], s2a);
      s2b = fmaf(w[OFF_W3 + o * NH + lane + 32], g3[warp][o], s2b);
    }
    const float d2a = s2a * gelu_grad(z2a), d2b = s2b * gelu_grad(z2b);
    g2[warp][lane] = d2a;
    g2[warp][lane + 32] = d2b;
    __syncwarp();
    for (int i = 0; i < NH; ++i) {
      atomicAdd(&gw[OFF_W2 + lane * NH + i], d2a * h1[warp][i]);
      atomicAdd(&gw[OFF_W2 + (lane + 32) * NH + i], d2b * h1[warp][i]);
    }
    atomicAdd(&gw[OFF_B2 + lane], d2a);
    atomicAdd(&gw[OFF_B2 + lane + 32], d2b);
    // layer 1: dh1 = W2^T dz2
    float s1a = 0.f, s1b = 0.f;
    for (int o = 0; o < NH; ++o) {
      s1a = fmaf(w[OFF_W2 + o * NH + lane], g2[warp][o], s1a);
      s1b = fmaf(w[OFF_W2 + o * NH + lane + 32], g2[warp][o], s1b);
    }
    const float d1a = s1a * gelu_grad(z1a), d1b = s1b * gelu_grad(z1b);
    for (int i = 0; i < NIN; ++i) {
      atomicAdd(&gw[OFF_W1 + lane * NIN + i], d1a * h0[warp][i]);
      atomicAdd(&gw[OFF_W1 + (lane + 32) * NIN + i], d1b * h0[warp][i]);
    }
    atomicAdd(&gw[OFF_B1 + lane], d1a);
    atomicAdd(&gw[OFF_B1 + lane + 32], d1b);
    __syncwarp();
  }
  if (lane == 0) lossw[warp] = loss;
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
    partial[(int64_t)blockIdx.x * NPARAM + i] = gw[i];
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int k = 0; k < WARPS; ++k) l += lossw[k];
    partial_loss[blockIdx.x] = l;
  }
}

__global__ void mlp_reduce_kernel(int nblocks, int batch, const float *partial,
                                  const float *partial_loss, float *grad, float *loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPARAM) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * NPARAM + i];
    grad[i] = s;
  }
  if (i == 0 && loss) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partial_loss[b];
    *loss = s / (float)batch;
  }
}

__global__ void mlp_adam_kernel(int n, float *theta, const float *grad, float *m, float *v,
                                float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 inference: weights and activations rounded to bf16, fp32 accumulation.
__global__ void __launch_bounds__(WARPS * 32) mlp_bf16_kernel(int n, const float *theta,
                                                               const float *X, float *pred) {
  __shared__ __nv_bfloat16 w[NPARAM + 1];
  __shared__ float h[WARPS][2][NH];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = __float2bfloat16_rn(theta[i]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto W = [&](int i) { return __bfloat162float(w[i]); };
  auto rb = [](float x) { return __bfloat162float(__float2bfloat16_rn(x)); };
  for (int smp = blockIdx.x * WARPS + warp; smp < n; smp += gridDim.x * WARPS) {
    float a0 = W(OFF_B1 + lane), a1 = W(OFF_B1 + lane + 32);
    for (int i = 0; i < NIN; ++i) {
      const float x = rb(X[(int64_t)smp * NIN + i]);
      a0 = fmaf(W(OFF_W1 + lane * NIN + i), x, a0);
      a1 = fmaf(W(OFF_W1 + (lane + 32) * NIN + i), x, a1);
    }
    h[warp][0][lane] = rb(gelu(a0));
    h[warp][0][lane + 32] = rb(gelu(a1));
    __syncwarp();
    for (int layer = 0; layer < 2; ++layer) {
      const int ow = layer == 0 ? OFF_W2 : OFF_W3, ob = layer == 0 ? OFF_B2 : OFF_B3;
      const float *hi = h[warp][layer & 1];
      a0 = W(ob + lane);
      a1 = W(ob + lane + 32);
      for (int i = 0; i < NH; ++i) {
        a0 = fmaf(W(ow + lane * NH + i), hi[i], a0);
        a1 = fmaf(W(ow + (lane + 32) * NH + i), hi[i], a1);
      }
      __syncwarp();
      h[warp][(layer + 1) & 1][lane] = rb(gelu(a0));
      h[warp][(layer + 1) & 1][lane + 32] = rb(gelu(a1));
      __syncwarp();
    }
    const float out = warp_sum(W(OFF_W4 + lane) * h[warp][0][lane] +
                               W(OFF_W4 + lane + 32) * h[warp][0][lane + 32]) +
                      W(OFF_B4);
    if (lane == 0) pred[smp] = out;
    __syncwarp();
  }
}

// argmin with ties to the smaller index, one block
__global__ void argmin_kernel(int n, const float *pred, int32_t *best) {
  __shared__ float bv[256];
  __shared__ int bi[256];
  float v = INFINITY;
  int idx = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float p = pred[i];
    if (p < v || (p == v && i < idx)) {
      v = p;
      idx = i;
    }
  }
  bv[threadIdx.x] = v;
  bi[threadIdx.x] = idx;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) {
      const float ov = bv[threadIdx.x + s];
      const int oi = bi[threadIdx.x + s];
      if (ov < bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = ov;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *best = bi[0] == 0x7fffffff ? -1 : bi[0];
}

int grid_for(int n) {
  const int b = (n + WARPS - 1) / WARPS;
  const int cap = state().sm_count > 0 ? state().sm_count * 4 : 512;
  return b < 1 ? 1 : (b < cap ? b : cap);
}

}  // namespace

// loaded model for hsumma_gemm's automatic choice
struct LoadedModel {
  bool loaded = false;
  float theta[NPARAM];
  float mean[NIN], stdv[NIN];
};
LoadedModel g_model;

const float *loaded_model(float *mean, float *stdv) {
  if (!g_model.loaded) return nullptr;
  for (int i = 0; i < NIN; ++i) {
    mean[i] = g_model.mean[i];
    stdv[i] = g_model.stdv[i];
  }
  return g_model.theta;
}

int mlp_pick_device(int n, const float *d_theta, const float *d_X, float *d_pred,
                    int32_t *d_best, cudaStream_t s) {
  mlp_bf16_kernel<<<grid_for(n), WARPS * 32, 0, s>>>(n, d_theta, d_X, d_pred);
  argmin_kernel<<<1, 256, 0, s>>>(n, d_pred, d_best);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSUMMA_OK : cuda_fail(e, "launch mlp pick");
}

// Scratch of hsumma_mlp_backward_noalloc: the per-block gradient partials
// (kNoAllocBlocks x NPARAM floats) followed by the per-block loss partials
// (kNoAllocBlocks floats), 18.6 MB in all.  It lives in the library's own
// device image, so every device that loads the library holds it until the
// process exits; nothing is allocated when the entry point runs.
constexpr int kNoAllocBlocks = (HSUMMA_MLP_NOALLOC_MAX_BATCH + WARPS - 1) / WARPS;
constexpr int kNoAllocDevices = 64;
static __device__ __align__(256) float g_noalloc_scratch[(size_t)kNoAllocBlocks * (NPARAM + 1)];

// Device address of g_noalloc_scratch on each device (host-side, filled on the
// first call made with that device current; emptied by hsumma_finalize, since a
// cudaDeviceReset in between leaves a stale address).
static std::mutex g_noalloc_mutex;
static float *g_noalloc_addr[kNoAllocDevices] = {};

void forget_noalloc_scratch() {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  for (auto &p : g_noalloc_addr) p = nullptr;
}

}  // namespace hs

using namespace hs;

extern "C" {

int hsumma_mlp_forward(int batch, const float *theta, const float *X, float *y, float *cache,
                       void *stream) {
  if (batch < 0 || (batch > 0 && (!theta || !X || !y))) {
    set_error("bad MLP arguments");
    return HSUMMA_ERR_ARG;
  }
  if (batch == 0) return HSUMMA_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  mlp_forward_kernel<<<grid_for(batch), WARPS * 32, 0, s>>>(batch, theta, X, y, cache);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSUMMA_OK : cuda_fail(e, "launch mlp forward");
}

int hsumma_mlp_backward(int batch, const float *theta, const float *X, const float *target,
                        float *grad, float *loss, void *stream) {
  if (batch <= 0 || !theta || !X || !target || !grad) {
    set_error("bad MLP arguments");
    return HSUMMA_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nb = grid_for(batch);
  // partial gradients of every block, reduced in block order (deterministic),
  // in a buffer of this call only, taken from and returned to the current
  // device's stream-ordered pool on `s`: calls on different devices, streams or
  // threads never share it, and growing it synchronises nothing
  float *partial = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&partial),
                                  (size_t)nb * (NPARAM + 1) * sizeof(float), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(mlp partials)");
  float *ploss = partial + (size_t)nb * NPARAM;
  const int smem = 2 * NPARAM * (int)sizeof(float);
  e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem);
  if (e == cudaSuccess) {
    mlp_backward_kernel<<<nb, WARPS * 32, smem, s>>>(batch, theta, X, target, partial, ploss);
    mlp_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(nb, batch, partial, ploss, grad,
                                                           loss);
    e = cudaGetLastError();
  }
  const cudaError_t ef = cudaFreeAsync(partial, s);
  if (e != cudaSuccess) return cuda_fail(e, "launch mlp backward");
  return ef == cudaSuccess ? HSUMMA_OK : cuda_fail(ef, "cudaFreeAsync(mlp partials)");
}

// Same gradient and loss as hsumma_mlp_backward, with the block partials kept
// in the fixed scratch above instead of a buffer grown with cudaMalloc.  Every
// slot the reduction reads (blocks 0..nb-1) is written by the backward kernel
// earlier in the same call, so nothing has to be cleared between calls.
int hsumma_mlp_backward_noalloc(int batch, const float *theta, const float *X,
                                const float *target, float *grad, float *loss, void *stream) {
  if (batch <= 0 || !theta || !X || !target || !grad) {
    set_error("bad MLP arguments");
    return HSUMMA_ERR_ARG;
  }
  if (batch > HSUMMA_MLP_NOALLOC_MAX_BATCH) {
    set_error("hsumma_mlp_backward_noalloc: batch %d exceeds its fixed scratch of "
              "HSUMMA_MLP_NOALLOC_MAX_BATCH = %d samples",
              batch, HSUMMA_MLP_NOALLOC_MAX_BATCH);
    return HSUMMA_ERR_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocDevices) {
    set_error("hsumma_mlp_backward_noalloc: device ordinal beyond 63");
    return HSUMMA_ERR_UNSUPPORTED;
  }
  float *partial = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void *addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(mlp scratch)");
      g_noalloc_addr[dev] = static_cast<float *>(addr);
    }
    partial = g_noalloc_addr[dev];
  }
  const int nb = grid_for(batch);  // <= ceil(batch / WARPS) <= kNoAllocBlocks
  float *ploss = partial + (size_t)kNoAllocBlocks * NPARAM;
  const int smem = 2 * NPARAM * (int)sizeof(float);
  e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mlp backward)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  mlp_backward_kernel<<<nb, WARPS * 32, smem, s>>>(batch, theta, X, target, partial, ploss);
  mlp_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(nb, batch, partial, ploss, grad, loss);
  e = cudaGetLastError();
  return e == cudaSuccess ? HSUMMA_OK : cuda_fail(e, "launch mlp backward (no-alloc)");
}

int hsumma_mlp_adam(int n, float *theta, const float *grad, float *m, float *v, int t, float lr,
                    float beta1, float beta2, float eps, void *stream) {
  if (n <= 0 || t < 1 || !theta || !grad || !m || !v) {
    set_error("bad Adam arguments");
    return HSUMMA_ERR_ARG;
  }
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  mlp_adam_kernel<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, theta, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSUMMA_OK : cuda_fail(e, "launch adam");
}

int hsumma_mlp_pick(int n, const float *theta, const float *X, float *pred, int32_t *best,
                    void *stream) {
  if (n <= 0 || !theta || !X || !pred || !best) {
    set_error("bad MLP arguments");
    return HSUMMA_ERR_ARG;
  }
  return mlp_pick_device(n, theta, X, pred, best, reinterpret_cast<cudaStream_t>(stream));
}

int hsumma_mlp_load(const float *theta, const float *mean, const float *stdv) {
  forget_model_range();
  if (!theta) {
    g_model.loaded = false;
    forget_choices();
    return HSUMMA_OK;
  }
  if (!mean || !stdv) {
    set_error("model needs feature means and standard deviations");
    return HSUMMA_ERR_ARG;
  }
  memcpy(g_model.theta, theta, sizeof(g_model.theta));
  memcpy(g_model.mean, mean, sizeof(g_model.mean));
  memcpy(g_model.stdv, stdv, sizeof(g_model.stdv));
  g_model.loaded = true;
  forget_choices();
  return HSUMMA_OK;
}

}  // extern "C"
