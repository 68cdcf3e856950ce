// Learned strategy selector: a 16 -> 64 -> 64 -> 3 MLP (ReLU,
// softmax, cross-entropy) with hand-written forward, backward and Adam
// kernels, trained on the GPU from the autotuner's labels. The paper's related
// work models the processing time of aggregation to choose a configuration
// (Sec. 7); here the model predicts the fastest strategy from the key sketch.
//
// Parameters are one float32 array of 5443 values:
//   W1 [16][64] at 0, b1 [64] at 1024, W2 [64][64] at 1088, b2 [64] at 5184,
//   W3 [64][3] at 5248, b3 [3] at 5440 (W[in][out], row-major).
// Inputs are standardised features (x - mean) / std.
// Classes: 0 = SMEM, 1 = GLOBAL, 2 = SORT.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "groupby.cuh"

namespace agg {

constexpr int kIn = 16, kH = 64, kOut = 3;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248, OFF_B3 = 5440;
constexpr int kParams = 5443;
constexpr int kParamsPad = 5448;
constexpr int kMlpThreads = 256;
constexpr int kMlpBatch = 256;  // samples per block
constexpr size_t kMlpSmem = sizeof(float) * ((size_t)kParamsPad + kMlpBatch * (kIn + 2 * kH + 4));

// One block handles up to kMlpBatch samples: forward pass, and with grads
// the backward pass with every reduction over the batch in a fixed order.
__global__ void __launch_bounds__(kMlpThreads) mlp_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ mean,
                                                          const float* __restrict__ stdv,
                                                          const float* __restrict__ X, const int32_t* __restrict__ y,
                                                          int n, float* __restrict__ probs, float* __restrict__ grads,
                                                          float* __restrict__ loss) {
  extern __shared__ __align__(16) float sm[];
  float* P = sm;
  float* x = P + kParamsPad;
  float* h1 = x + kMlpBatch * kIn;
  float* h2 = h1 + kMlpBatch * kH;
  float* dz = h2 + kMlpBatch * kH;  // [B][4]
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * kMlpBatch;
  const int B = min(kMlpBatch, n - b0);
  if (B <= 0) return;
  for (int i = tid; i < kParams; i += kMlpThreads) P[i] = params[i];
  for (int i = tid; i < B * kIn; i += kMlpThreads) {
    const int f = i % kIn;
    float v = X[(size_t)b0 * kIn + i];
    if (mean) v = (v - mean[f]) / stdv[f];
    x[i] = v;
  }
  __syncthreads();
  for (int i = tid; i < B * kH; i += kMlpThreads) {
    const int b = i / kH, j = i % kH;
    float acc = P[OFF_B1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) acc = fmaf(x[b * kIn + k], P[OFF_W1 + k * kH + j], acc);
    h1[i] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  for (int i = tid; i < B * kH; i += kMlpThreads) {
    const int b = i / kH, j = i % kH;
    float acc = P[OFF_B2 + j];
#pragma unroll 8
    for (int k = 0; k < kH; ++k) acc = fmaf(h1[b * kH + k], P[OFF_W2 + k * kH + j], acc);
    h2[i] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  float my_loss = 0.f;
  for (int b = tid; b < B; b += kMlpThreads) {
    float z[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      float acc = P[OFF_B3 + o];
      for (int k = 0; k < kH; ++k) acc = fmaf(h2[b * kH + k], P[OFF_W3 + k * kOut + o], acc);
      z[o] = acc;
    }
    const float zm = fmaxf(z[0], fmaxf(z[1], z[2]));
    float e[kOut], se = 0.f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      e[o] = expf(z[o] - zm);
      se += e[o];
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      const float p = e[o] / se;
      if (probs) probs[(size_t)(b0 + b) * kOut + o] = p;
      if (grads) dz[b * 4 + o] = (p - (y[b0 + b] == o ? 1.f : 0.f)) / (float)B;
    }
    if (grads) my_loss += -(z[y[b0 + b]] - zm - logf(se));
  }
  if (!grads) return;
  __shared__ float red[kMlpThreads / 32];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
  if ((tid & 31) == 0) red[tid >> 5] = my_loss;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int i = 0; i < kMlpThreads / 32; ++i) t += red[i];
    *loss = t / (float)B;
  }
  // layer 3: dW3[k][o] = sum_b h2[b][k] dz[b][o], db3[o] = sum_b dz[b][o]
  for (int i = tid; i < kH * kOut + kOut; i += kMlpThreads) {
    float acc = 0.f;
    if (i < kH * kOut) {
      const int k = i / kOut, o = i % kOut;
      for (int b = 0; b < B; ++b) acc = fmaf(h2[b * kH + k], dz[b * 4 + o], acc);
      grads[OFF_W3 + i] = acc;
    } else {
      const int o = i - kH * kOut;
      for (int b = 0; b < B; ++b) acc += dz[b * 4 + o];
      grads[OFF_B3 + o] = acc;
    }
  }
  __syncthreads();
  // dh2 = (dz W3^T) * relu'(h2), in place of h2
  for (int i = tid; i < B * kH; i += kMlpThreads) {
    const int b = i / kH, k = i % kH;
    float acc = 0.f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) acc = fmaf(dz[b * 4 + o], P[OFF_W3 + k * kOut + o], acc);
    h2[i] = h2[i] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  // layer 2: dW2[k][j] = sum_b h1[b][k] dh2[b][j], db2[j] = sum_b dh2[b][j]
  for (int i = tid; i < kH * kH + kH; i += kMlpThreads) {
    float acc = 0.f;
    if (i < kH * kH) {
      const int k = i / kH, j = i % kH;
      for (int b = 0; b < B; ++b) acc = fmaf(h1[b * kH + k], h2[b * kH + j], acc);
      grads[OFF_W2 + i] = acc;
    } else {
      const int j = i - kH * kH;
      for (int b = 0; b < B; ++b) acc += h2[b * kH + j];
      grads[OFF_B2 + j] = acc;
    }
  }
  __syncthreads();
  // dh1 = (dh2 W2^T) * relu'(h1), in place of h1
  for (int i = tid; i < B * kH; i += kMlpThreads) {
    const int b = i / kH, k = i % kH;
    float acc = 0.f;
#pragma unroll 8
    for (int j = 0; j < kH; ++j) acc = fmaf(h2[b * kH + j], P[OFF_W2 + k * kH + j], acc);
    h1[i] = h1[i] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  // layer 1: dW1[i][j] = sum_b x[b][i] dh1[b][j], db1[j] = sum_b dh1[b][j]
  for (int i = tid; i < kIn * kH + kH; i += kMlpThreads) {
    float acc = 0.f;
    if (i < kIn * kH) {
      const int f = i / kH, j = i % kH;
      for (int b = 0; b < B; ++b) acc = fmaf(x[b * kIn + f], h1[b * kH + j], acc);
      grads[OFF_W1 + i] = acc;
    } else {
      const int j = i - kIn * kH;
      for (int b = 0; b < B; ++b) acc += h1[b * kH + j];
      grads[OFF_B1 + j] = acc;
    }
  }
}

// Adam (Kingma and Ba, ICLR 2015), bias-corrected, step t >= 1.
__global__ void mlp_adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int64_t t, float lr, float b1, float b2, float eps) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void gather_rows(const float* __restrict__ X, const int32_t* __restrict__ y,
                            const int32_t* __restrict__ idx, int B, float* __restrict__ Xb,
                            int32_t* __restrict__ yb) {
  for (int i = threadIdx.x; i < B * kIn; i += blockDim.x) Xb[i] = X[(size_t)idx[i / kIn] * kIn + i % kIn];
  for (int i = threadIdx.x; i < B; i += blockDim.x) yb[i] = y[idx[i]];
}

static agg_status mlp_attr() {
  static bool set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && set[dev]) return AGG_OK;
  AGG_CUDA_TRY(cudaFuncSetAttribute(mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem));
  if (dev < 64) set[dev] = true;
  return AGG_OK;
}

static agg_status mlp_launch(const float* params, const float* mean, const float* stdv, const float* X,
                             const int32_t* y, int n, float* probs, float* grads, float* loss, cudaStream_t s) {
  agg_status st = mlp_attr();
  if (st != AGG_OK) return st;
  const int grid = grads ? 1 : (n + kMlpBatch - 1) / kMlpBatch;
  PhaseTimer pt(AGG_PHASE_MLP, s);
  mlp_kernel<<<grid, kMlpThreads, kMlpSmem, s>>>(params, mean, stdv, X, y, n, probs, grads, loss);
  note_launch();
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

// ---------------------------------------------------------------------------
// The installed selector (per device): weights and feature standardisation.
// ---------------------------------------------------------------------------
struct Selector {
  bool ok = false;
  float* dev = nullptr;  // params | mean | std (device)
  std::vector<float> host;
};
static std::mutex g_sel_mu;
static Selector g_sel[64];

static Selector* selector_for_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  return &g_sel[dev];
}

// Sketch and, if a selector is installed, run the network on the device
// features; one read-back for both. *strategy = -1 when no selector is set.
agg_status sketch_and_select(const uint32_t* keys, int64_t n, int vdt, uint32_t ops, uint64_t offset,
                             cudaStream_t s, float* feat, int* strategy) {
  *strategy = -1;
  agg_status st = AGG_OK;
  float* fd = (float*)stream_scratch(s, 4096, &st);
  if (!fd) return st;
  // features at float 512 and probabilities at float 544 of the stream scratch
  // (past the reduce ticket; that region only ever holds transient values)
  float* fdev = fd + 512;
  float* pdev = fd + 544;
  st = sketch_launch(keys, n, vdt, ops, offset, fdev, s);
  if (st != AGG_OK) return st;
  float* sel = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_sel_mu);
    Selector* S = selector_for_device();
    if (S && S->ok) sel = S->dev;
  }
  if (sel) {
    st = mlp_launch(sel, sel + kParamsPad, sel + kParamsPad + kIn, fdev, nullptr, 1, pdev, nullptr, nullptr, s);
    if (st != AGG_OK) return st;
  }
  float* hb = (float*)stream_pinned(s, 256, &st);
  if (!hb) return st;
  AGG_CUDA_TRY(cudaMemcpyAsync(hb, fdev, 40 * sizeof(float), cudaMemcpyDeviceToHost, s));
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(feat, hb, F_COUNT * sizeof(float));
  if (sel) {
    const float* p = hb + 32;
    int best = 0;
    for (int o = 1; o < kOut; ++o)
      if (p[o] > p[best]) best = o;
    *strategy = best == 0 ? AGG_STRAT_SMEM : best == 1 ? AGG_STRAT_GLOBAL : AGG_STRAT_SORT;
  }
  return AGG_OK;
}

// Batched sketch, then (with a selector installed) the network on all the
// sketches in one launch.
agg_status batch_select(const SketchJob* jobs_dev, int nq, float* feat_dev, float* probs_dev, cudaStream_t s,
                        bool* have_probs) {
  *have_probs = false;
  agg_status st = sketch_batch_launch(jobs_dev, nq, feat_dev, s);
  if (st != AGG_OK) return st;
  float* sel = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_sel_mu);
    Selector* S = selector_for_device();
    if (S && S->ok) sel = S->dev;
  }
  if (!sel) return AGG_OK;
  st = mlp_launch(sel, sel + kParamsPad, sel + kParamsPad + kIn, feat_dev, nullptr, nq, probs_dev, nullptr, nullptr, s);
  if (st == AGG_OK) *have_probs = true;
  return st;
}

// Strategy from host features (used by the host-fed path): one tiny launch.
int select_learned(const float* feat, bool* ok) {
  *ok = false;
  float* sel = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_sel_mu);
    Selector* S = selector_for_device();
    if (S && S->ok) sel = S->dev;
  }
  if (!sel) return AGG_STRAT_GLOBAL;
  agg_status st = AGG_OK;
  cudaStream_t s = nullptr;
  float* fd = (float*)stream_scratch(s, 4096, &st);
  if (!fd) return AGG_STRAT_GLOBAL;
  float* fdev = fd + 512;
  float* pdev = fd + 544;
  if (cudaMemcpy(fdev, feat, F_COUNT * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return AGG_STRAT_GLOBAL;
  if (mlp_launch(sel, sel + kParamsPad, sel + kParamsPad + kIn, fdev, nullptr, 1, pdev, nullptr, nullptr, s) != AGG_OK)
    return AGG_STRAT_GLOBAL;
  float p[kOut];
  if (cudaMemcpy(p, pdev, sizeof(p), cudaMemcpyDeviceToHost) != cudaSuccess) return AGG_STRAT_GLOBAL;
  int best = 0;
  for (int o = 1; o < kOut; ++o)
    if (p[o] > p[best]) best = o;
  *ok = true;
  return best == 0 ? AGG_STRAT_SMEM : best == 1 ? AGG_STRAT_GLOBAL : AGG_STRAT_SORT;
}

}  // namespace agg

using namespace agg;

extern "C" int agg_mlp_param_count(void) { return kParams; }

extern "C" agg_status agg_mlp_forward(const float* params_dev, const float* mean_dev, const float* std_dev,
                                      const float* x_dev, int n, float* probs_dev, void* stream) {
  clear_error();
  AGG_CHECK_ARG(params_dev && x_dev && probs_dev && n >= 0, "invalid arguments");
  AGG_CHECK_ARG((mean_dev == nullptr) == (std_dev == nullptr), "mean and std must both be given or both be null");
  if (n == 0) return AGG_OK;
  return mlp_launch(params_dev, mean_dev, std_dev, x_dev, nullptr, n, probs_dev, nullptr, nullptr,
                    (cudaStream_t)stream);
}

extern "C" agg_status agg_mlp_grad(const float* params_dev, const float* mean_dev, const float* std_dev,
                                   const float* x_dev, const int32_t* y_dev, int n, float* grads_dev,
                                   float* loss_dev, void* stream) {
  clear_error();
  AGG_CHECK_ARG(params_dev && x_dev && y_dev && grads_dev && loss_dev, "null pointer");
  AGG_CHECK_ARG(n >= 1 && n <= kMlpBatch, "batch must hold 1..%d samples", kMlpBatch);
  AGG_CHECK_ARG((mean_dev == nullptr) == (std_dev == nullptr), "mean and std must both be given or both be null");
  return mlp_launch(params_dev, mean_dev, std_dev, x_dev, y_dev, n, nullptr, grads_dev, loss_dev,
                    (cudaStream_t)stream);
}

extern "C" agg_status agg_mlp_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev,
                                   int64_t t, float lr, float beta1, float beta2, float eps, void* stream) {
  clear_error();
  AGG_CHECK_ARG(params_dev && grads_dev && m_dev && v_dev && t >= 1, "invalid arguments");
  mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params_dev, grads_dev, m_dev, v_dev, t,
                                                                           lr, beta1, beta2, eps);
  note_launch();
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

// Mini-batch training on the device: each epoch visits the samples in a
// seeded SplitMix64 Fisher-Yates order, in batches of `batch` (<= 256).
extern "C" agg_status agg_mlp_train(float* params_dev, float* m_dev, float* v_dev, const float* mean_dev,
                                    const float* std_dev, const float* x_dev, const int32_t* y_dev, int n,
                                    int epochs, int batch, float lr, uint64_t seed, int64_t t0,
                                    float* epoch_loss_host, void* stream) {
  clear_error();
  AGG_CHECK_ARG(params_dev && m_dev && v_dev && x_dev && y_dev && n >= 1 && epochs >= 0, "invalid arguments");
  AGG_CHECK_ARG(batch >= 1 && batch <= kMlpBatch, "batch must be in 1..%d", kMlpBatch);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  const int nb = (n + batch - 1) / batch;
  float *grads = nullptr, *xb = nullptr, *losses = nullptr;
  int32_t *yb = nullptr, *idx = nullptr;
  {
    void* blk = nullptr;
    const size_t b0 = 256 * ((sizeof(float) * kParamsPad + 255) / 256), b1 = 256 * ((sizeof(float) * kMlpBatch * kIn + 255) / 256),
                 b2 = 256 * ((sizeof(int32_t) * kMlpBatch + 255) / 256), b3 = 256 * ((sizeof(int32_t) * (size_t)n + 255) / 256);
    AGG_CUDA_TRY(dev_malloc_async(&blk, b0 + b1 + b2 + b3 + sizeof(float) * (size_t)nb, s));
    grads = (float*)blk;
    xb = (float*)((char*)blk + b0);
    yb = (int32_t*)((char*)blk + b0 + b1);
    idx = (int32_t*)((char*)blk + b0 + b1 + b2);
    losses = (float*)((char*)blk + b0 + b1 + b2 + b3);
  }
  uint64_t st64 = seed;
  auto next = [&]() {  // SplitMix64
    uint64_t z = (st64 += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  int64_t t = t0;
  agg_status st = AGG_OK;
  std::vector<float> hl(nb);
  for (int ep = 0; ep < epochs && st == AGG_OK; ++ep) {
    for (int i = n - 1; i > 0; --i) {
      const int j = (int)(next() % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    if (cudaMemcpyAsync(idx, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("index upload failed");
      st = AGG_ERR_CUDA;
      break;
    }
    for (int bi = 0; bi < nb && st == AGG_OK; ++bi) {
      const int B = std::min(batch, n - bi * batch);
      gather_rows<<<1, 256, 0, s>>>(x_dev, y_dev, idx + (size_t)bi * batch, B, xb, yb);
      note_launch();
      st = mlp_launch(params_dev, mean_dev, std_dev, xb, yb, B, nullptr, grads, losses + bi, s);
      if (st != AGG_OK) break;
      mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params_dev, grads, m_dev, v_dev, ++t, lr, 0.9f, 0.999f,
                                                            1e-8f);
      note_launch();
    }
    if (st == AGG_OK && epoch_loss_host) {
      if (cudaMemcpyAsync(hl.data(), losses, sizeof(float) * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("loss read-back failed");
        st = AGG_ERR_CUDA;
        break;
      }
      double sum = 0;
      for (int bi = 0; bi < nb; ++bi) sum += hl[bi] * std::min(batch, n - bi * batch);
      epoch_loss_host[ep] = (float)(sum / n);
    }
  }
  cudaFreeAsync(grads, s);  // the one block holding all of the scratch
  if (st == AGG_OK) AGG_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

extern "C" agg_status agg_selector_set(const float* params_host, const float* mean_host, const float* std_host) {
  clear_error();
  AGG_CHECK_ARG(params_host && mean_host && std_host, "null pointer");
  for (int i = 0; i < kIn; ++i) AGG_CHECK_ARG(std_host[i] > 0.f, "std[%d] must be positive", i);
  std::lock_guard<std::mutex> lk(g_sel_mu);
  Selector* S = selector_for_device();
  AGG_CHECK_ARG(S != nullptr, "device index out of range");
  if (!S->dev) AGG_CUDA_TRY(dev_malloc((void**)&S->dev, sizeof(float) * (kParamsPad + 2 * kIn)));
  S->host.assign(kParamsPad + 2 * kIn, 0.f);
  std::memcpy(S->host.data(), params_host, sizeof(float) * kParams);
  std::memcpy(S->host.data() + kParamsPad, mean_host, sizeof(float) * kIn);
  std::memcpy(S->host.data() + kParamsPad + kIn, std_host, sizeof(float) * kIn);
  AGG_CUDA_TRY(cudaMemcpy(S->dev, S->host.data(), sizeof(float) * S->host.size(), cudaMemcpyHostToDevice));
  S->ok = true;
  return AGG_OK;
}

extern "C" void agg_selector_clear(void) {
  std::lock_guard<std::mutex> lk(g_sel_mu);
  Selector* S = selector_for_device();
  if (S) S->ok = false;
}

extern "C" int agg_selector_installed(void) {
  std::lock_guard<std::mutex> lk(g_sel_mu);
  Selector* S = selector_for_device();
  return S && S->ok ? 1 : 0;
}
