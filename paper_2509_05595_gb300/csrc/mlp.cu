// The learned proposal's network: a per-edge MLP 16 -> 64 -> 64 -> 1 (ReLU,
// ReLU, logistic) with BF16 weights and FP32 accumulation, and its training
// (weighted binary cross-entropy, Adam).  No counterpart in the paper: it
// predicts which collapses the intersection check of Section 5.2 would undo
// (Section 5.3), so that they can be deferred instead of tested.
//
// Parameters, flat (fp32 master copy, bf16 working copy, same layout):
//   W1 [16][64] at 0, b1 [64] at 1024, W2 [64][64] at 1088, b2 [64] at 5184,
//   W3 [64] at 5248, b3 at 5312; 5313 in all.  W[i][j] maps input i to
//   output j.
//
// Inputs are standardised first, x' = (x - mu) * inv_sd (fp32, per feature;
// identity by default), so that the BF16 first layer never has to absorb the
// features' offsets and scales.
//
// Forward: one thread per sample, weights staged in shared memory as fp32
// (converted from bf16 once per block).  Backward: one block per chunk of 64
// samples keeps the activations of the chunk in shared memory and reduces
// the weight gradients over the chunk (outer products summed in a fixed
// order); each block accumulates its partial over a grid-stride of chunks,
// and a second kernel sums the per-block partials in block order, so the
// gradient is deterministic.
#include <cuda_bf16.h>

#include "common.cuh"

namespace pamo {
namespace {

constexpr int kIn = PAMO_MLP_IN, kH = PAMO_MLP_HIDDEN;
constexpr int oW1 = 0, oB1 = kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH, kParams = oB3 + 1;
static_assert(kParams == PAMO_MLP_PARAMS, "parameter layout");

constexpr int kChunk = 64;        // samples per backward chunk
constexpr int kGradBlocks = 304;  // fixed grid of the backward pass (2 per SM)

__device__ __forceinline__ float sigmoidf_(float x) {
  // 1 / (1 + e^-x) from the exponential; for large |x| it saturates to 0 / 1
  return 1.0f / (1.0f + __expf(-x));
}

// stable log(1 + e^x)
__device__ __forceinline__ float softplusf_(float x) {
  return x > 0.f ? x + log1pf(__expf(-x)) : log1pf(__expf(x));
}

// weights as fp32, then the 2 x 16 standardisation (mu, inv_sd) after them
__device__ __forceinline__ void load_weights(const __nv_bfloat16* __restrict__ pb,
                                             const float* __restrict__ norm, float* w) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = __bfloat162float(pb[i]);
  for (int i = threadIdx.x; i < 2 * kIn; i += blockDim.x) w[kParams + i] = norm[i];
  __syncthreads();
}

__device__ __forceinline__ void standardise(const float* __restrict__ w, float* x) {
#pragma unroll
  for (int i = 0; i < kIn; i++) x[i] = (x[i] - w[kParams + i]) * w[kParams + kIn + i];
}

// logit of one sample; h1 (post-ReLU) and a2 (post-ReLU) optionally stored
template <bool kStore>
__device__ __forceinline__ float forward_one(const float* __restrict__ w, const float* x, float* h1s,
                                             float* a2s) {
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; j++) h1[j] = w[oB1 + j];
#pragma unroll
  for (int i = 0; i < kIn; i++) {
    const float xi = x[i];
#pragma unroll
    for (int j = 0; j < kH; j++) h1[j] = fmaf(xi, w[oW1 + i * kH + j], h1[j]);
  }
#pragma unroll
  for (int j = 0; j < kH; j++) {
    h1[j] = fmaxf(h1[j], 0.f);
    if (kStore) h1s[j] = h1[j];
  }
  float out = w[oB3];
#pragma unroll
  for (int j0 = 0; j0 < kH; j0 += 16) {
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = w[oB2 + j0 + k];
#pragma unroll  // constant indices keep h1 in registers
    for (int i = 0; i < kH; i++) {
      const float hi = h1[i];
#pragma unroll
      for (int k = 0; k < 16; k++) acc[k] = fmaf(hi, w[oW2 + i * kH + j0 + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const float a = fmaxf(acc[k], 0.f);
      if (kStore) a2s[j0 + k] = a;
      out = fmaf(a, w[oW3 + j0 + k], out);
    }
  }
  return out;
}

__global__ void __launch_bounds__(kBlock) k_mlp_forward(const __nv_bfloat16* __restrict__ pb,
                                                        const float* __restrict__ norm,
                                                        const float* __restrict__ X,
                                                        const int* n_dev, int64_t n_host,
                                                        float* __restrict__ prob) {
  __shared__ float w[kParams + 2 * kIn];
  const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
  if ((int64_t)blockIdx.x * blockDim.x >= n) return;  // no sample: skip the weight load
  load_weights(pb, norm, w);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    float x[kIn];
    const float4* xv = reinterpret_cast<const float4*>(X + kIn * s);
#pragma unroll
    for (int q = 0; q < kIn / 4; q++) {
      const float4 v = xv[q];
      x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
    }
    standardise(w, x);
    prob[s] = sigmoidf_(forward_one<false>(w, x, nullptr, nullptr));
  }
}

// Weighted BCE over n samples: loss_s = -(pw y log p + (1 - y) log(1 - p)),
// averaged; per-block partial gradients (and loss) into part[block][kParams+1].
__global__ void __launch_bounds__(kChunk) k_mlp_grad(const __nv_bfloat16* __restrict__ pb,
                                                     const float* __restrict__ norm,
                                                     const float* __restrict__ X,
                                                     const float* __restrict__ y, int64_t n,
                                                     float pos_weight, float* __restrict__ part) {
  extern __shared__ float sm[];
  float* w = sm;                       // kParams + 2 kIn (weights, standardisation)
  float* g = w + kParams + 2 * kIn;    // kParams + 1 (the loss last)
  float* Xs = g + kParams + 1;         // kChunk x kIn
  float* H1 = Xs + kChunk * kIn;       // kChunk x kH
  float* A2 = H1 + kChunk * kH;        // kChunk x kH
  float* D2 = A2 + kChunk * kH;        // kChunk x kH
  float* D1 = D2 + kChunk * kH;        // kChunk x kH
  float* d3 = D1 + kChunk * kH;        // kChunk
  float* ls = d3 + kChunk;             // kChunk: per-sample loss
  load_weights(pb, norm, w);
  for (int i = threadIdx.x; i <= kParams; i += blockDim.x) g[i] = 0.f;
  const float inv_n = 1.0f / (float)n;
  const int t = threadIdx.x;
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < n; c0 += (int64_t)gridDim.x * kChunk) {
    const int64_t s = c0 + t;
    const bool ok = s < n;
    // forward of this thread's sample (rows past n are zero inputs with zero
    // error, so they add nothing)
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; i++) x[i] = ok ? X[kIn * s + i] : 0.f;
    standardise(w, x);
#pragma unroll
    for (int i = 0; i < kIn; i++) {
      if (!ok) x[i] = 0.f;
      Xs[t * kIn + i] = x[i];
    }
    const float z = forward_one<true>(w, x, H1 + t * kH, A2 + t * kH);
    float delta = 0.f, loss = 0.f;
    if (ok) {
      const float yy = y[s], p = sigmoidf_(z);
      // d/dz of -(pw y log p + (1-y) log(1-p)) = pw y (p - 1) + (1 - y) p
      delta = (pos_weight * yy * (p - 1.f) + (1.f - yy) * p) * inv_n;
      loss = (pos_weight * yy * softplusf_(-z) + (1.f - yy) * softplusf_(z)) * inv_n;
    }
    d3[t] = delta;
    ls[t] = loss;
    // back through layers 3 and 2 for this sample
#pragma unroll 8
    for (int j = 0; j < kH; j++) D2[t * kH + j] = A2[t * kH + j] > 0.f ? delta * w[oW3 + j] : 0.f;
    for (int i = 0; i < kH; i++) {
      float acc = 0.f;
#pragma unroll 8
      for (int j = 0; j < kH; j++) acc = fmaf(w[oW2 + i * kH + j], D2[t * kH + j], acc);
      D1[t * kH + i] = H1[t * kH + i] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // weight gradients of the chunk, each entry summed over samples in order
    for (int e = t; e <= kParams; e += blockDim.x) {
      float acc = 0.f;
      if (e < oB1) {  // W1[i][j] += x_i * d1_j
        const int i = e / kH, j = e % kH;
        for (int k = 0; k < kChunk; k++) acc = fmaf(Xs[k * kIn + i], D1[k * kH + j], acc);
      } else if (e < oW2) {
        const int j = e - oB1;
        for (int k = 0; k < kChunk; k++) acc += D1[k * kH + j];
      } else if (e < oB2) {  // W2[i][j] += h1_i * d2_j
        const int i = (e - oW2) / kH, j = (e - oW2) % kH;
        for (int k = 0; k < kChunk; k++) acc = fmaf(H1[k * kH + i], D2[k * kH + j], acc);
      } else if (e < oW3) {
        const int j = e - oB2;
        for (int k = 0; k < kChunk; k++) acc += D2[k * kH + j];
      } else if (e < oB3) {  // W3[j] += a2_j * d3
        const int j = e - oW3;
        for (int k = 0; k < kChunk; k++) acc = fmaf(A2[k * kH + j], d3[k], acc);
      } else if (e == oB3) {
        for (int k = 0; k < kChunk; k++) acc += d3[k];
      } else {  // the loss of the chunk
        for (int k = 0; k < kChunk; k++) acc += ls[k];
      }
      g[e] += acc;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i <= kParams; i += blockDim.x)
    part[(int64_t)blockIdx.x * (kParams + 1) + i] = g[i];
}

// sum of the per-block partials in block order (deterministic)
__global__ void k_mlp_grad_reduce(const float* __restrict__ part, int nblocks,
                                  float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kParams) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; b++) s += part[(int64_t)b * (kParams + 1) + i];
  grad[i] = s;
}

// Adam (Kingma & Ba 2015) on the fp32 master weights; refreshes the bf16 copy
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g,
                           float* __restrict__ m, float* __restrict__ v,
                           __nv_bfloat16* __restrict__ pb, float lr, float b1, float b2,
                           float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
  p[i] = pi;
  pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kParams) pb[i] = __float2bfloat16_rn(p[i]);
}

// Input standardisation from the training data: per feature, the mean and
// the population standard deviation over n rows, in float64 with a fixed
// reduction order (deterministic), two passes (mean, then squared
// deviations).  kNormBlocks blocks of 16 x 16 threads: thread (r, j) sums
// feature j over rows b + kNormBlocks (r + 16 k); the 16 row lanes, then the
// blocks, are summed in order.
constexpr int kNormBlocks = 256;

__global__ void __launch_bounds__(256) k_norm_pass(const float* __restrict__ X, int64_t n,
                                                   const double* __restrict__ mean,
                                                   double* __restrict__ part) {
  __shared__ double acc[16][kIn];
  const int j = threadIdx.x % kIn, r = threadIdx.x / kIn;
  const double m = mean ? mean[j] : 0.0;
  double s = 0.0;
  for (int64_t i = blockIdx.x + (int64_t)kNormBlocks * r; i < n; i += (int64_t)kNormBlocks * 16) {
    const double x = (double)X[kIn * i + j];
    s = mean ? s + (x - m) * (x - m) : s + x;
  }
  acc[r][j] = s;
  __syncthreads();
  if (r == 0) {
    double t = 0.0;
    for (int q = 0; q < 16; q++) t += acc[q][j];
    part[blockIdx.x * kIn + j] = t;
  }
}

// sums the block partials in block order; first pass: mean; second: the
// standardisation (mu, 1/sd), sd below 1e-6 taken as 1
__global__ void k_norm_final(const double* __restrict__ part, int64_t n, double* __restrict__ mean,
                             float* __restrict__ norm, int second) {
  const int j = threadIdx.x;
  if (j >= kIn) return;
  double t = 0.0;
  for (int b = 0; b < kNormBlocks; b++) t += part[b * kIn + j];
  if (!second) {
    mean[j] = t / (double)n;
  } else {
    const double sd = sqrt(t / (double)n);
    norm[j] = (float)mean[j];
    norm[kIn + j] = sd < 1e-6 ? 1.0f : (float)(1.0 / sd);
  }
}

size_t grad_smem_bytes() {
  return sizeof(float) *
         ((size_t)2 * kParams + 2 * kIn + 1 + kChunk * kIn + 4 * kChunk * kH + 2 * kChunk);
}

}  // namespace

}  // namespace pamo

using namespace pamo;

struct pamo_mlp {
  float* norm = nullptr;           // [2][16] input standardisation (mu, 1/sd)
  float* p = nullptr;              // fp32 master weights
  __nv_bfloat16* pb = nullptr;     // bf16 working copy
  float* m = nullptr;              // Adam moments
  float* v = nullptr;
  float* grad = nullptr;           // last gradient, loss at [kParams]
  float* part = nullptr;           // per-block partials
  int64_t step = 0;
};

namespace pamo {

pamo_status mlp_forward_dev(const pamo_mlp* m, const float* X, const int* n_dev, float* prob,
                            int64_t n_host, cudaStream_t st) {
  static const int g = occ_grid(k_mlp_forward);
  k_mlp_forward<<<g, kBlock, 0, st>>>(m->pb, m->norm, X, n_dev, n_host, prob); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo

extern "C" {

pamo_status pamo_mlp_create(pamo_mlp** out) {
  if (!out) {
    set_error("out is NULL");
    return PAMO_EINVAL;
  }
  pamo_mlp* m = new pamo_mlp();
  cudaError_t e = cudaMalloc(&m->p, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * 2 * kIn);
  if (e == cudaSuccess) {
    float id[2 * kIn];
    for (int i = 0; i < kIn; i++) {
      id[i] = 0.f;
      id[kIn + i] = 1.f;
    }
    e = cudaMemcpy(m->norm, id, sizeof(id), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->pb, sizeof(__nv_bfloat16) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->m, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->v, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * (kParams + 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->part, sizeof(float) * (kParams + 1) * kGradBlocks);
  if (e == cudaSuccess) e = cudaMemset(m->p, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(m->pb, 0, sizeof(__nv_bfloat16) * kParams);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(m->grad, 0, sizeof(float) * (kParams + 1));
  if (e != cudaSuccess) {
    pamo_mlp_destroy(m);
    return cuda_fail(e, "pamo_mlp_create");
  }
  *out = m;
  return PAMO_OK;
}

void pamo_mlp_destroy(pamo_mlp* m) {
  if (!m) return;
  cudaFree(m->norm);
  cudaFree(m->p);
  cudaFree(m->pb);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->grad);
  cudaFree(m->part);
  delete m;
}

pamo_status pamo_mlp_set_params(pamo_mlp* m, const float* h_params) {
  if (!m || !h_params) {
    set_error("model and parameters required");
    return PAMO_EINVAL;
  }
  PAMO_CUDA(cudaMemcpy(m->p, h_params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
  k_to_bf16<<<(kParams + 255) / 256, 256>>>(m->p, m->pb); note_launch();
  PAMO_CUDA(cudaGetLastError());
  PAMO_CUDA(cudaMemset(m->m, 0, sizeof(float) * kParams));
  PAMO_CUDA(cudaMemset(m->v, 0, sizeof(float) * kParams));
  PAMO_CUDA(cudaDeviceSynchronize());
  m->step = 0;
  return PAMO_OK;
}

pamo_status pamo_mlp_set_input_norm(pamo_mlp* m, const float* h_mu, const float* h_sd) {
  if (!m || !h_mu || !h_sd) {
    set_error("model, mu and sd required");
    return PAMO_EINVAL;
  }
  float v[2 * kIn];
  for (int i = 0; i < kIn; i++) {
    if (!(h_sd[i] > 0.f)) {
      set_error("standard deviations must be > 0");
      return PAMO_EINVAL;
    }
    v[i] = h_mu[i];
    v[kIn + i] = 1.0f / h_sd[i];
  }
  PAMO_CUDA(cudaMemcpy(m->norm, v, sizeof(v), cudaMemcpyHostToDevice));
  return PAMO_OK;
}

pamo_status pamo_mlp_fit_input_norm(pamo_mlp* m, const float* d_X, int64_t n, void* stream) {
  if (!m || !d_X || n <= 0) {
    set_error("model and at least one feature row required");
    return PAMO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* buf = nullptr;  // [kNormBlocks][16] partials, then [16] means
  PAMO_CUDA(cudaMallocAsync((void**)&buf, sizeof(double) * (kNormBlocks + 1) * kIn, st));
  double* mean = buf + kNormBlocks * kIn;
  k_norm_pass<<<kNormBlocks, 256, 0, st>>>(d_X, n, nullptr, buf); note_launch();
  k_norm_final<<<1, 32, 0, st>>>(buf, n, mean, m->norm, 0); note_launch();
  k_norm_pass<<<kNormBlocks, 256, 0, st>>>(d_X, n, mean, buf); note_launch();
  k_norm_final<<<1, 32, 0, st>>>(buf, n, mean, m->norm, 1); note_launch();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(buf, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "pamo_mlp_fit_input_norm");
  return PAMO_OK;
}

pamo_status pamo_mlp_get_params(const pamo_mlp* m, float* h_params, uint16_t* h_bf16) {
  if (!m) {
    set_error("model required");
    return PAMO_EINVAL;
  }
  if (h_params)
    PAMO_CUDA(cudaMemcpy(h_params, m->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
  if (h_bf16)
    PAMO_CUDA(cudaMemcpy(h_bf16, m->pb, sizeof(uint16_t) * kParams, cudaMemcpyDeviceToHost));
  return PAMO_OK;
}

pamo_status pamo_mlp_forward(const pamo_mlp* m, const float* d_X, int64_t n, float* d_prob,
                             void* stream) {
  if (!m || n < 0 || (n > 0 && (!d_X || !d_prob))) {
    set_error("bad forward arguments");
    return PAMO_EINVAL;
  }
  if (n == 0) return PAMO_OK;
  return mlp_forward_dev(m, d_X, nullptr, d_prob, n, (cudaStream_t)stream);
}

pamo_status pamo_mlp_grad(pamo_mlp* m, const float* d_X, const float* d_y, int64_t n,
                          float pos_weight, void* stream, float* h_loss) {
  if (!m || n <= 0 || !d_X || !d_y || !(pos_weight > 0.f)) {
    set_error("bad gradient arguments");
    return PAMO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  static bool attr = false;
  const size_t smem = grad_smem_bytes();
  if (!attr) {
    PAMO_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = true;
  }
  k_mlp_grad<<<kGradBlocks, kChunk, smem, st>>>(m->pb, m->norm, d_X, d_y, n, pos_weight,
                                                 m->part); note_launch();
  k_mlp_grad_reduce<<<(kParams + 1 + 255) / 256, 256, 0, st>>>(m->part, kGradBlocks, m->grad); note_launch();
  PAMO_CUDA(cudaGetLastError());
  if (h_loss) {
    PAMO_CUDA(cudaMemcpyAsync(h_loss, m->grad + kParams, sizeof(float), cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaStreamSynchronize(st));
  }
  return PAMO_OK;
}

pamo_status pamo_mlp_get_grad(const pamo_mlp* m, float* h_grad) {
  if (!m || !h_grad) {
    set_error("model and output required");
    return PAMO_EINVAL;
  }
  PAMO_CUDA(cudaDeviceSynchronize());
  PAMO_CUDA(cudaMemcpy(h_grad, m->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
  return PAMO_OK;
}

pamo_status pamo_mlp_adam_step(pamo_mlp* m, float lr, float beta1, float beta2, float eps,
                               void* stream) {
  if (!m || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f)) {
    set_error("bad Adam arguments");
    return PAMO_EINVAL;
  }
  m->step++;
  const float c1 = 1.f - powf(beta1, (float)m->step), c2 = 1.f - powf(beta2, (float)m->step);
  k_mlp_adam<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      m->p, m->grad, m->m, m->v, m->pb, lr, beta1, beta2, eps, c1, c2); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // extern "C"
