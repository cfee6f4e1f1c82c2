// hmat_rank.cu -- the learned rank proposal: a 12 -> 64 -> 64 -> 1 MLP (ReLU) that predicts a far
// block's eps-rank (as log2(1 + rank)) from features of its sum-expression. Weights are held in
// FP16 for the forward pass with FP32 accumulation; training keeps FP32 master weights and
// updates them with Adam. One training step = forward + backward over the whole batch (mean
// squared error) + the Adam update; the host captures a step once in a CUDA graph and replays
// it for the requested number of epochs.
#include <cmath>
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hm {

// parameter layout (floats): W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3[1]
constexpr int F = RANK_FEATURES, H = 64;
constexpr int O_W1 = 0, O_B1 = O_W1 + H * F, O_W2 = O_B1 + H, O_B2 = O_W2 + H * H, O_W3 = O_B2 + H, O_B3 = O_W3 + H;
static_assert(O_B3 + 1 == RANK_PARAMS, "parameter layout");

constexpr int RT = 256;          // threads per block
constexpr int RW = RT / 32;      // warps per block

// Forward (and, with grad != nullptr, backward) of a chunk of samples per block, warp per
// sample. x: count x F (already normalised), y: targets (log2(1 + rank)); weights in FP16.
// Shared memory holds the weights in the layouts that let a warp's lanes read consecutive
// words (W1 and W2 transposed for the forward pass, W2 as stored for the backward pass) and the
// gradients transposed the same way; the block's gradient sum is added to grad at the end.
struct MlpSmem {
  float W1T[F * H];   // W1T[i * H + j] = W1[j][i]
  float W2T[H * H];   // W2T[k * H + j] = W2[j][k]
  float W2[H * H];    // W2[j * H + k]
  float b1[H], b2[H], w3[H], b3;
  float G1T[F * H], G2T[H * H], Gb1[H], Gb2[H], Gw3[H], Gb3;
  float act[RW][2 * H];
  float lsum[RW];
};

__global__ void __launch_bounds__(RT) k_mlp(const __half *w16, const float *x, const float *y, int count, float *out,
                                            float *grad, float *loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem &S = *(MlpSmem *)smem_raw;
  for (int o = threadIdx.x; o < H * F; o += RT) {
    const int j = o / F, i = o - j * F;
    S.W1T[i * H + j] = __half2float(w16[O_W1 + o]);
    S.G1T[o] = 0.f;
  }
  for (int o = threadIdx.x; o < H * H; o += RT) {
    const int j = o / H, k = o - j * H;
    const float wv = __half2float(w16[O_W2 + o]);
    S.W2[o] = wv;
    S.W2T[k * H + j] = wv;
    S.G2T[o] = 0.f;
  }
  for (int j = threadIdx.x; j < H; j += RT) {
    S.b1[j] = __half2float(w16[O_B1 + j]);
    S.b2[j] = __half2float(w16[O_B2 + j]);
    S.w3[j] = __half2float(w16[O_W3 + j]);
    S.Gb1[j] = S.Gb2[j] = S.Gw3[j] = 0.f;
  }
  if (threadIdx.x == 0) {
    S.b3 = __half2float(w16[O_B3]);
    S.Gb3 = 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *act = S.act[warp];
  float lacc = 0.f;
  const float inv = 1.f / (float)count;
  for (int s = blockIdx.x * RW + warp; s < count; s += gridDim.x * RW) {
    const float *xs = x + (int64_t)s * F;
    float xv[F];
#pragma unroll
    for (int i = 0; i < F; i++) xv[i] = xs[i];
    float h1[2], h2[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {  // layer 1: lane owns units lane, lane + 32
      const int j = lane + 32 * u;
      float a = S.b1[j];
#pragma unroll
      for (int i = 0; i < F; i++) a += S.W1T[i * H + j] * xv[i];
      h1[u] = fmaxf(a, 0.f);
      act[j] = h1[u];
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; u++) {  // layer 2
      const int j = lane + 32 * u;
      float a = S.b2[j];
      for (int k = 0; k < H; k++) a += S.W2T[k * H + j] * act[k];
      h2[u] = fmaxf(a, 0.f);
    }
    float o = S.w3[lane] * h2[0] + S.w3[lane + 32] * h2[1];
    for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
    o += S.b3;
    if (out && lane == 0) out[s] = o;
    if (grad) {
      const float e = o - y[s];
      lacc += e * e;
      const float dout = 2.f * e * inv;
      if (lane == 0) atomicAdd(&S.Gb3, dout);
      float dh2[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int j = lane + 32 * u;
        atomicAdd(&S.Gw3[j], dout * h2[u]);
        dh2[u] = h2[u] > 0.f ? dout * S.w3[j] : 0.f;
        atomicAdd(&S.Gb2[j], dh2[u]);
        for (int k = 0; k < H; k++) atomicAdd(&S.G2T[k * H + j], dh2[u] * act[k]);  // dW2[j][k]
      }
      __syncwarp();
      act[H + lane] = dh2[0];
      act[H + lane + 32] = dh2[1];
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 2; u++) {  // dh1[k] = sum_j W2[j][k] dh2[j]
        const int k = lane + 32 * u;
        float d = 0.f;
        for (int j = 0; j < H; j++) d += S.W2[j * H + k] * act[H + j];
        d = h1[u] > 0.f ? d : 0.f;
        atomicAdd(&S.Gb1[k], d);
#pragma unroll
        for (int i = 0; i < F; i++) atomicAdd(&S.G1T[i * H + k], d * xv[i]);
      }
    }
    __syncwarp();
  }
  if (grad) {
    if (lane == 0) S.lsum[warp] = lacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < RW; w++) t += S.lsum[w];
      atomicAdd(loss, t * inv);
    }
    for (int o = threadIdx.x; o < H * F; o += RT) {
      const int j = o / F, i = o - j * F;
      atomicAdd(&grad[O_W1 + o], S.G1T[i * H + j]);
    }
    for (int o = threadIdx.x; o < H * H; o += RT) {
      const int j = o / H, k = o - j * H;
      atomicAdd(&grad[O_W2 + o], S.G2T[k * H + j]);
    }
    for (int j = threadIdx.x; j < H; j += RT) {
      atomicAdd(&grad[O_B1 + j], S.Gb1[j]);
      atomicAdd(&grad[O_B2 + j], S.Gb2[j]);
      atomicAdd(&grad[O_W3 + j], S.Gw3[j]);
    }
    if (threadIdx.x == 0) atomicAdd(&grad[O_B3], S.Gb3);
  }
}

static cudaError_t set_mlp_smem() {
  return raise_smem_limit(k_mlp, sizeof(MlpSmem));
}

// Adam on the FP32 masters, then the FP16 copies used by the forward pass
__global__ void k_adam(float *w, __half *w16, float *m, float *v, const float *grad, float lr, float b1, float b2,
                       float eps, int *step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = *step + 1;
  if (i < RANK_PARAMS) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
    w16[i] = __float2half(w[i]);
  }
}

__global__ void k_step_inc(int *step) { *step += 1; }

__global__ void k_to_half(const float *w, __half *w16, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w16[i] = __float2half(w[i]);
}

static int mlp_grid(int count) {
  const int g = (count + RW * 4 - 1) / (RW * 4);  // about 4 samples per warp
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

cudaError_t launch_mlp_forward(const void *w16, const float *x, int count, float *out, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  cudaError_t e = set_mlp_smem();
  if (e != cudaSuccess) return e;
  k_mlp<<<mlp_grid(count), RT, sizeof(MlpSmem), s>>>((const __half *)w16, x, nullptr, count, out, nullptr, nullptr);
  return cudaGetLastError();
}

// stream work only (the kernel's shared-memory attribute is set by the caller), so that it can
// be captured into a graph
static cudaError_t mlp_grad_ops(const void *w16, const float *x, const float *y, int count, float *grad, float *loss,
                                cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(grad, 0, sizeof(float) * RANK_PARAMS, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  k_mlp<<<mlp_grid(count), RT, sizeof(MlpSmem), s>>>((const __half *)w16, x, y, count, nullptr, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const void *w16, const float *x, const float *y, int count, float *grad, float *loss,
                            cudaStream_t s) {
  cudaError_t e = set_mlp_smem();
  if (e != cudaSuccess) return e;
  return mlp_grad_ops(w16, x, y, count, grad, loss, s);
}

cudaError_t launch_to_half(const float *w, void *w16, cudaStream_t s) {
  k_to_half<<<(RANK_PARAMS + 255) / 256, 256, 0, s>>>(w, (__half *)w16, RANK_PARAMS);
  return cudaGetLastError();
}

cudaError_t mlp_train(float *w, void *w16, const float *x, const float *y, int count, int epochs, float lr,
                      cudaStream_t s, float *final_loss) {
  float *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
  int *step = nullptr;
  cudaError_t e = cudaSuccess;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaFree(m);
    cudaFree(v);
    cudaFree(grad);
    cudaFree(loss);
    cudaFree(step);
  };
  if ((e = cudaMalloc(&m, sizeof(float) * RANK_PARAMS)) || (e = cudaMalloc(&v, sizeof(float) * RANK_PARAMS)) ||
      (e = cudaMalloc(&grad, sizeof(float) * RANK_PARAMS)) || (e = cudaMalloc(&loss, sizeof(float))) ||
      (e = cudaMalloc(&step, sizeof(int)))) {
    cleanup();
    return e;
  }
  if ((e = set_mlp_smem())) { cleanup(); return e; }
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) { cleanup(); return e; }
  cudaEvent_t ready;
  if ((e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming))) { cleanup(); return e; }
  cudaMemsetAsync(m, 0, sizeof(float) * RANK_PARAMS, s);
  cudaMemsetAsync(v, 0, sizeof(float) * RANK_PARAMS, s);
  cudaMemsetAsync(step, 0, sizeof(int), s);
  launch_to_half(w, w16, s);
  cudaEventRecord(ready, s);
  cudaStreamWaitEvent(cs, ready, 0);
  cudaEventDestroy(ready);
  // one step, captured once and replayed
  if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal))) { cleanup(); return e; }
  mlp_grad_ops(w16, x, y, count, grad, loss, cs);
  k_adam<<<(RANK_PARAMS + 255) / 256, 256, 0, cs>>>(w, (__half *)w16, m, v, grad, lr, 0.9f, 0.999f, 1e-8f, step);
  k_step_inc<<<1, 1, 0, cs>>>(step);
  if ((e = cudaStreamEndCapture(cs, &graph))) { cleanup(); return e; }
  if ((e = cudaGraphInstantiate(&exec, graph, 0))) { cleanup(); return e; }
  for (int ep = 0; ep < epochs; ep++)
    if ((e = cudaGraphLaunch(exec, cs))) { cleanup(); return e; }
  if (final_loss) {
    mlp_grad_ops(w16, x, y, count, grad, loss, cs);
    cudaMemcpyAsync(final_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, cs);
  }
  e = cudaStreamSynchronize(cs);
  cleanup();
  return e;
}

// ---------------------------------------------------------------------------------------
// Gradient without device allocation. Every device buffer of the call lives in the fixed
// array below: features (RANKGRAD_NOALLOC_MAX x F), targets, the gradient and the loss.
// (RANKGRAD_NOALLOC_MAX * 13 + RANK_PARAMS + 1 floats, about 0.87 MB per device.)
// ---------------------------------------------------------------------------------------

constexpr size_t NOALLOC_FLOATS = (size_t)RANKGRAD_NOALLOC_MAX * (F + 1) + RANK_PARAMS + 1;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

struct Standardise {
  float mean[F], dev[F];
};

// in place: x <- (x - mean) / dev per feature (FP32, as the allocating call does on the host);
// y <- log2(1 + max(y, 0)), evaluated in FP64 and rounded to FP32 like the allocating call's
// targets
__global__ void k_standardise(float *x, float *y, int count, Standardise sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count * F) {
    const int k = i % F;
    x[i] = (x[i] - sd.mean[k]) / sd.dev[k];
  }
  if (i < count) y[i] = (float)log2(1.0 + fmax((double)y[i], 0.0));
}

// The scratch array's device address on the current device. It is looked up on every call
// (cudaGetSymbolAddress allocates nothing): a cached address would go stale if the device's
// primary context were reset and the module reloaded. The network kernel's shared-memory limit
// is set on every call for the same reason.
static cudaError_t noalloc_scratch(float **out) {
  float *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if ((e = set_mlp_smem()) != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

cudaError_t mlp_grad_noalloc(const void *w16, const float *mean, const float *dev, const float *features,
                             const float *ranks, int count, float *grad, float *loss, cudaStream_t s) {
  if (count < 1 || count > RANKGRAD_NOALLOC_MAX) return cudaErrorInvalidValue;
  float *base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return e;
  float *x = base, *y = x + (size_t)RANKGRAD_NOALLOC_MAX * F;
  float *g = y + RANKGRAD_NOALLOC_MAX, *l = g + RANK_PARAMS;
  Standardise sd;
  for (int k = 0; k < F; k++) {
    sd.mean[k] = mean[k];
    sd.dev[k] = dev[k];
  }
  if ((e = cudaMemcpyAsync(x, features, sizeof(float) * F * count, cudaMemcpyHostToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(y, ranks, sizeof(float) * count, cudaMemcpyHostToDevice, s))) return e;
  k_standardise<<<(count * F + 255) / 256, 256, 0, s>>>(x, y, count, sd);
  if ((e = cudaGetLastError())) return e;
  // the gradient and the loss are accumulated with atomics: mlp_grad_ops first sets both to zero
  if ((e = mlp_grad_ops(w16, x, y, count, g, l, s))) return e;
  if ((e = cudaMemcpyAsync(grad, g, sizeof(float) * RANK_PARAMS, cudaMemcpyDeviceToHost, s))) return e;
  if (loss && (e = cudaMemcpyAsync(loss, l, sizeof(float), cudaMemcpyDeviceToHost, s))) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace hm
