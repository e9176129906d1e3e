// hmat_mlp.cu -- training and evaluation of the rank predictor on the GPU.
//
// Gradients of the mean squared error of the network's output against
// log(1 + rank) come from the library's own backward kernel: each CTA takes a
// chunk of 64 samples, runs the forward pass with the BF16-rounded weights in
// shared memory, back-propagates in FP32 and adds its chunk's gradient to the
// global FP32 gradient once per parameter.  Adam (Kingma and Ba 2015) updates
// the FP32 masters, then their BF16 copy is refreshed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hmat.h"
#include "hmat_mlp.cuh"

namespace hm_internal {
int ctx_device(const hmat_ctx* c);
cudaStream_t ctx_stream(const hmat_ctx* c);
void set_last_error(const char* msg);
}  // namespace hm_internal

struct hmat_mlp {
  hmat_ctx* ctx = nullptr;
  float* master = nullptr;       // FP32 masters
  __nv_bfloat16* w = nullptr;    // BF16 copy used by every forward pass
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  float* loss = nullptr;
  int64_t steps = 0;
};

namespace {

#define MLP_CHUNK 64

struct MlpFail {
  hmat_status code;
  std::string msg;
};

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw MlpFail{e == cudaErrorMemoryAllocation ? HMAT_ERR_NOMEM : HMAT_ERR_CUDA,
                  std::string(what) + ": " + cudaGetErrorString(e)};
}

template <class F>
hmat_status mlp_guard(F f) {
  try {
    f();
    return HMAT_OK;
  } catch (const MlpFail& e) {
    hm_internal::set_last_error(e.msg.c_str());
    return e.code;
  }
}

__global__ void to_bf16(const float* a, __nv_bfloat16* b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// Gradient of sum_s (f(x_s) - y_s)^2 / count over the chunk of this CTA.
__global__ void __launch_bounds__(256) mlp_grad(const __nv_bfloat16* Wb, const float* X, const float* Y, int count,
                                                float inv_count, float* grad, float* loss) {
  extern __shared__ float sm[];
  float* W1 = sm;                              // 384
  float* B1 = W1 + HM_MLP_H * HM_MLP_IN;       // 64
  float* W2 = B1 + HM_MLP_H;                   // 4096
  float* B2 = W2 + HM_MLP_H * HM_MLP_H;        // 64
  float* W3 = B2 + HM_MLP_H;                   // 64
  float* Xs = W3 + HM_MLP_H + 4;               // 64 x 6
  float* H1 = Xs + MLP_CHUNK * HM_MLP_IN;      // 64 x 64 (sample-major)
  float* H2 = H1 + MLP_CHUNK * HM_MLP_H;
  float* D2 = H2 + MLP_CHUNK * HM_MLP_H;
  float* D1 = D2 + MLP_CHUNK * HM_MLP_H;
  float* dO = D1 + MLP_CHUNK * HM_MLP_H;       // 64
  int tid = threadIdx.x;
  int s0 = blockIdx.x * MLP_CHUNK;
  int ns = count - s0 < MLP_CHUNK ? count - s0 : MLP_CHUNK;
  for (int i = tid; i < HM_MLP_NPARAM - 1; i += blockDim.x) sm[i] = __bfloat162float(Wb[i]);
  float b3 = __bfloat162float(Wb[HM_MLP_B3]);
  for (int i = tid; i < MLP_CHUNK * HM_MLP_IN; i += blockDim.x) Xs[i] = (i / HM_MLP_IN) < ns ? X[(int64_t)s0 * HM_MLP_IN + i] : 0.f;
  __syncthreads();
  for (int idx = tid; idx < MLP_CHUNK * HM_MLP_H; idx += blockDim.x) {
    int s = idx / HM_MLP_H, o = idx % HM_MLP_H;
    float a = B1[o];
    for (int i = 0; i < HM_MLP_IN; ++i) a += W1[o * HM_MLP_IN + i] * Xs[s * HM_MLP_IN + i];
    H1[idx] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < MLP_CHUNK * HM_MLP_H; idx += blockDim.x) {
    int s = idx / HM_MLP_H, o = idx % HM_MLP_H;
    float a = B2[o];
    for (int i = 0; i < HM_MLP_H; ++i) a += W2[o * HM_MLP_H + i] * H1[s * HM_MLP_H + i];
    H2[idx] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  if (tid < MLP_CHUNK) {
    float r = 0.f;
    if (tid < ns) {
      float a = b3;
      for (int i = 0; i < HM_MLP_H; ++i) a += W3[i] * H2[tid * HM_MLP_H + i];
      r = a - Y[s0 + tid];
      atomicAdd(loss, r * r * inv_count);
    }
    dO[tid] = 2.f * r * inv_count;
  }
  __syncthreads();
  for (int idx = tid; idx < MLP_CHUNK * HM_MLP_H; idx += blockDim.x) {
    int s = idx / HM_MLP_H, o = idx % HM_MLP_H;
    D2[idx] = H2[idx] > 0.f ? dO[s] * W3[o] : 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < MLP_CHUNK * HM_MLP_H; idx += blockDim.x) {
    int s = idx / HM_MLP_H, i = idx % HM_MLP_H;
    float a = 0.f;
    for (int o = 0; o < HM_MLP_H; ++o) a += D2[s * HM_MLP_H + o] * W2[o * HM_MLP_H + i];
    D1[idx] = H1[idx] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // parameter gradients: sums over the chunk's samples
  for (int p = tid; p < HM_MLP_NPARAM; p += blockDim.x) {
    float g = 0.f;
    if (p < HM_MLP_B1) {
      int o = p / HM_MLP_IN, i = p % HM_MLP_IN;
      for (int s = 0; s < MLP_CHUNK; ++s) g += D1[s * HM_MLP_H + o] * Xs[s * HM_MLP_IN + i];
    } else if (p < HM_MLP_W2) {
      int o = p - HM_MLP_B1;
      for (int s = 0; s < MLP_CHUNK; ++s) g += D1[s * HM_MLP_H + o];
    } else if (p < HM_MLP_B2) {
      int o = (p - HM_MLP_W2) / HM_MLP_H, i = (p - HM_MLP_W2) % HM_MLP_H;
      for (int s = 0; s < MLP_CHUNK; ++s) g += D2[s * HM_MLP_H + o] * H1[s * HM_MLP_H + i];
    } else if (p < HM_MLP_W3) {
      int o = p - HM_MLP_B2;
      for (int s = 0; s < MLP_CHUNK; ++s) g += D2[s * HM_MLP_H + o];
    } else if (p < HM_MLP_B3) {
      int i = p - HM_MLP_W3;
      for (int s = 0; s < MLP_CHUNK; ++s) g += dO[s] * H2[s * HM_MLP_H + i];
    } else {
      for (int s = 0; s < MLP_CHUNK; ++s) g += dO[s];
    }
    atomicAdd(grad + p, g);
  }
}

const size_t GRAD_SMEM =
    sizeof(float) * (HM_MLP_NPARAM + 4 + MLP_CHUNK * HM_MLP_IN + 4 * MLP_CHUNK * HM_MLP_H + MLP_CHUNK);

__global__ void adam_step(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                          float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + 1e-8f);
}

__global__ void mlp_eval(const __nv_bfloat16* W, const float* X, int count, float* out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= count) return;
  float x[HM_MLP_IN];
  for (int i = 0; i < HM_MLP_IN; ++i) x[i] = X[(int64_t)warp * HM_MLP_IN + i];
  float y = hm::mlp_forward_warp(W, x);
  if ((threadIdx.x & 31) == 0) out[warp] = y;
}

struct Dev {
  void* p = nullptr;
  explicit Dev(size_t b) { ck(cudaMalloc(&p, b ? b : 16), "cudaMalloc"); }
  ~Dev() { cudaFree(p); }
};

void refresh_bf16(hmat_mlp* M, cudaStream_t st) {
  to_bf16<<<(HM_MLP_NPARAM + 255) / 256, 256, 0, st>>>(M->master, M->w, HM_MLP_NPARAM);
  ck(cudaGetLastError(), "to_bf16");
}

// gradient and loss of one batch into M->grad / M->loss
void batch_grad(hmat_mlp* M, const float* dX, const float* dY, int count, cudaStream_t st) {
  ck(cudaMemsetAsync(M->grad, 0, HM_MLP_NPARAM * sizeof(float), st), "memset");
  ck(cudaMemsetAsync(M->loss, 0, sizeof(float), st), "memset");
  int blocks = (count + MLP_CHUNK - 1) / MLP_CHUNK;
  mlp_grad<<<blocks, 256, GRAD_SMEM, st>>>(M->w, dX, dY, count, 1.f / (float)count, M->grad, M->loss);
  ck(cudaGetLastError(), "mlp_grad");
}

// counter-based uniform in (0, 1) (SplitMix64 finaliser)
double unif(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) + 0.5) / 9007199254740992.0;
}

}  // namespace

namespace hm_internal {
const void* mlp_weights(const hmat_mlp* M) { return M ? (const void*)M->w : nullptr; }
}  // namespace hm_internal

extern "C" {

hmat_status hmat_mlp_create(hmat_ctx* ctx, uint64_t seed, hmat_mlp** out) {
  return mlp_guard([&] {
    if (!ctx || !out) throw MlpFail{HMAT_ERR_ARG, "hmat_mlp_create: null argument"};
    ck(cudaSetDevice(hm_internal::ctx_device(ctx)), "cudaSetDevice");
    cudaStream_t st = hm_internal::ctx_stream(ctx);
    auto* M = new hmat_mlp();
    M->ctx = ctx;
    size_t fb = HM_MLP_NPARAM * sizeof(float);
    ck(cudaMalloc(&M->master, fb), "cudaMalloc");
    ck(cudaMalloc(&M->w, HM_MLP_NPARAM * sizeof(__nv_bfloat16)), "cudaMalloc");
    ck(cudaMalloc(&M->m, fb), "cudaMalloc");
    ck(cudaMalloc(&M->v, fb), "cudaMalloc");
    ck(cudaMalloc(&M->grad, fb), "cudaMalloc");
    ck(cudaMalloc(&M->loss, sizeof(float)), "cudaMalloc");
    ck(cudaFuncSetAttribute(mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM), "smem");
    // He-uniform initial weights (bounds sqrt(6 / fan_in)), zero biases
    std::vector<float> p(HM_MLP_NPARAM, 0.f);
    for (int i = 0; i < HM_MLP_H * HM_MLP_IN; ++i)
      p[HM_MLP_W1 + i] = (float)((2.0 * unif(seed, i) - 1.0) * std::sqrt(6.0 / HM_MLP_IN));
    for (int i = 0; i < HM_MLP_H * HM_MLP_H; ++i)
      p[HM_MLP_W2 + i] = (float)((2.0 * unif(seed, 1000 + i) - 1.0) * std::sqrt(6.0 / HM_MLP_H));
    for (int i = 0; i < HM_MLP_H; ++i)
      p[HM_MLP_W3 + i] = (float)((2.0 * unif(seed, 9000 + i) - 1.0) * std::sqrt(6.0 / HM_MLP_H));
    ck(cudaMemcpyAsync(M->master, p.data(), fb, cudaMemcpyHostToDevice, st), "copy");
    ck(cudaMemsetAsync(M->m, 0, fb, st), "memset");
    ck(cudaMemsetAsync(M->v, 0, fb, st), "memset");
    refresh_bf16(M, st);
    ck(cudaStreamSynchronize(st), "sync");
    *out = M;
  });
}

hmat_status hmat_mlp_destroy(hmat_mlp* M) {
  if (M) {
    cudaFree(M->master);
    cudaFree(M->w);
    cudaFree(M->m);
    cudaFree(M->v);
    cudaFree(M->grad);
    cudaFree(M->loss);
    delete M;
  }
  return HMAT_OK;
}

hmat_status hmat_mlp_get_params(const hmat_mlp* M, float* out) {
  return mlp_guard([&] {
    if (!M || !out) throw MlpFail{HMAT_ERR_ARG, "null argument"};
    ck(cudaMemcpy(out, M->master, HM_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost), "copy");
  });
}

hmat_status hmat_mlp_set_params(hmat_mlp* M, const float* in) {
  return mlp_guard([&] {
    if (!M || !in) throw MlpFail{HMAT_ERR_ARG, "null argument"};
    cudaStream_t st = hm_internal::ctx_stream(M->ctx);
    ck(cudaMemcpyAsync(M->master, in, HM_MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    refresh_bf16(M, st);
    ck(cudaStreamSynchronize(st), "sync");
  });
}

hmat_status hmat_mlp_forward(const hmat_mlp* M, int64_t count, const float* X, float* y) {
  return mlp_guard([&] {
    if (!M || (count > 0 && (!X || !y))) throw MlpFail{HMAT_ERR_ARG, "null argument"};
    if (count <= 0) return;
    cudaStream_t st = hm_internal::ctx_stream(M->ctx);
    Dev dX(count * HM_MLP_IN * sizeof(float)), dY(count * sizeof(float));
    ck(cudaMemcpyAsync(dX.p, X, count * HM_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    int blocks = (int)((count * 32 + 255) / 256);
    mlp_eval<<<blocks, 256, 0, st>>>(M->w, (const float*)dX.p, (int)count, (float*)dY.p);
    ck(cudaGetLastError(), "mlp_eval");
    ck(cudaMemcpyAsync(y, dY.p, count * sizeof(float), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
  });
}

hmat_status hmat_mlp_grad(hmat_mlp* M, int64_t count, const float* X, const float* y, float* loss, float* grad) {
  return mlp_guard([&] {
    if (!M || count <= 0 || !X || !y || !loss || !grad) throw MlpFail{HMAT_ERR_ARG, "bad arguments"};
    cudaStream_t st = hm_internal::ctx_stream(M->ctx);
    Dev dX(count * HM_MLP_IN * sizeof(float)), dY(count * sizeof(float));
    ck(cudaMemcpyAsync(dX.p, X, count * HM_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    ck(cudaMemcpyAsync(dY.p, y, count * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    batch_grad(M, (const float*)dX.p, (const float*)dY.p, (int)count, st);
    ck(cudaMemcpyAsync(grad, M->grad, HM_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
  });
}

hmat_status hmat_mlp_train(hmat_mlp* M, int64_t count, const float* X, const float* y, int epochs, int batch,
                           float lr, uint64_t seed, float* final_loss) {
  return mlp_guard([&] {
    if (!M || count <= 0 || !X || !y || epochs < 1 || batch < 1 || !(lr > 0.f))
      throw MlpFail{HMAT_ERR_ARG, "hmat_mlp_train: bad arguments"};
    cudaStream_t st = hm_internal::ctx_stream(M->ctx);
    // one seeded shuffle per epoch on the host, batches copied in that order
    std::vector<int64_t> order((size_t)count);
    std::vector<float> Xb((size_t)count * HM_MLP_IN), yb((size_t)count);
    Dev dX(count * HM_MLP_IN * sizeof(float)), dY(count * sizeof(float));
    for (int ep = 0; ep < epochs; ++ep) {
      for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
      for (int64_t i = count - 1; i > 0; --i) {  // Fisher-Yates
        int64_t j = (int64_t)(unif(seed + (uint64_t)ep * 1315423911ull, (uint64_t)i) * (double)(i + 1));
        if (j > i) j = i;
        std::swap(order[(size_t)i], order[(size_t)j]);
      }
      for (int64_t i = 0; i < count; ++i) {
        std::memcpy(&Xb[(size_t)i * HM_MLP_IN], &X[order[(size_t)i] * HM_MLP_IN], HM_MLP_IN * sizeof(float));
        yb[(size_t)i] = y[order[(size_t)i]];
      }
      ck(cudaMemcpyAsync(dX.p, Xb.data(), Xb.size() * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
      ck(cudaMemcpyAsync(dY.p, yb.data(), yb.size() * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
      for (int64_t b0 = 0; b0 < count; b0 += batch) {
        int nb = (int)std::min<int64_t>(batch, count - b0);
        batch_grad(M, (const float*)dX.p + b0 * HM_MLP_IN, (const float*)dY.p + b0, nb, st);
        ++M->steps;
        float c1 = 1.f - std::pow(0.9f, (float)M->steps), c2 = 1.f - std::pow(0.999f, (float)M->steps);
        adam_step<<<(HM_MLP_NPARAM + 255) / 256, 256, 0, st>>>(M->master, M->grad, M->m, M->v, HM_MLP_NPARAM, lr,
                                                               0.9f, 0.999f, c1, c2);
        ck(cudaGetLastError(), "adam_step");
        refresh_bf16(M, st);
      }
      // the next epoch's shuffle rewrites the host staging buffers
      ck(cudaStreamSynchronize(st), "sync");
    }
    if (final_loss) {
      // loss of the trained network on the whole set
      Dev dX2(count * HM_MLP_IN * sizeof(float)), dY2(count * sizeof(float));
      ck(cudaMemcpyAsync(dX2.p, X, count * HM_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
      ck(cudaMemcpyAsync(dY2.p, y, count * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
      batch_grad(M, (const float*)dX2.p, (const float*)dY2.p, (int)count, st);
      ck(cudaMemcpyAsync(final_loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st), "copy");
    }
    ck(cudaStreamSynchronize(st), "sync");
  });
}

}  // extern "C"
