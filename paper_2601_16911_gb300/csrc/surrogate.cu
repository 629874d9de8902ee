// The surrogate sensor network: its training on the GPU (forward, backward, deterministic
// gradient reduction and Adam, all hand-written: BF16-rounded inputs and weights, FP32
// arithmetic), the packing of its weights into tensor-core fragments, stand-alone
// inference (the same warp-level MMA routine the fused stage kernel runs), the features
// mode of the stage kernel that produces training data, and attaching a trained network
// to a mesh.  The paper has no learned component; the network estimates its sensor
// gamma_e (eq. gamma) from cell-vertex data, and the plain sensor decides wherever the
// network's confidence is low.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "cvweno_internal.cuh"
#include "mlp_mma.cuh"

using namespace cvw;

namespace {

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }
inline cvweno_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CVWENO_OK : CVWENO_ERR_CUDA; }

constexpr int kGradThreads = 256;
constexpr int kSub = 64;            // samples per shared-memory sub-batch
constexpr int kMaxGradBlocks = 304; // 2 x 152 SMs
constexpr float kLam = 0.1f, kTau = 0.05f;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// tanh-form GELU and its derivative with the accurate tanhf (training path)
__device__ __forceinline__ float gelu_acc(float x, float& dgelu) {
  const float c = 0.7978845608028654f;
  const float u = c * fmaf(0.044715f * x * x, x, x);
  const float t = tanhf(u);
  dgelu = 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * c * fmaf(3.0f * 0.044715f, x * x, 1.0f);
  return 0.5f * x * (1.0f + t);
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }
__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x))); }

// Shared-memory layout of the gradient kernel (floats).
struct GradLayout {
  static constexpr int W = 0;                        // kMlpParams: W rounded to bf16, biases FP32
  static constexpr int X = (kMlpParams + 3) / 4 * 4; // [kSub][12]
  static constexpr int Z1 = X + kSub * kMlpIn;       // [kSub][64] z1, then dz1
  static constexpr int A1 = Z1 + kSub * 64;          // [kSub][64]
  static constexpr int Z2 = A1 + kSub * 64;          // [kSub][64] z2, then dz2
  static constexpr int A2 = Z2 + kSub * 64;          // [kSub][64]
  static constexpr int DO = A2 + kSub * 64;          // [kSub][2] outputs, then their gradient
  static constexpr int LS = DO + kSub * 2;           // [kSub] per-sample loss
  static constexpr int FLOATS = LS + kSub;
};

// Forward and backward over samples [begin, end) of this block's share of the batch;
// writes the block's summed gradient (already divided by the batch size n) and loss.
__global__ void __launch_bounds__(kGradThreads)
    mlp_grad_kernel(const float* __restrict__ params, const float* __restrict__ X, const float* __restrict__ y,
                    int64_t n, int64_t per_block, float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ __align__(16) float sm[];
  using L = GradLayout;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMlpParams; i += kGradThreads) {
    const bool is_w = i < kMlpOffB1 || (i >= kMlpOffW2 && i < kMlpOffB2) || (i >= kMlpOffW3 && i < kMlpOffB3);
    sm[L::W + i] = is_w ? bf16r(params[i]) : params[i];
  }
  const float* W1 = sm + L::W + kMlpOffW1;
  const float* B1 = sm + L::W + kMlpOffB1;
  const float* W2 = sm + L::W + kMlpOffW2;
  const float* B2 = sm + L::W + kMlpOffB2;
  const float* W3 = sm + L::W + kMlpOffW3;
  const float* B3 = sm + L::W + kMlpOffB3;
  float* xs = sm + L::X;
  float* z1 = sm + L::Z1;
  float* a1 = sm + L::A1;
  float* z2 = sm + L::Z2;
  float* a2 = sm + L::A2;
  float* dout = sm + L::DO;
  float* ls = sm + L::LS;
  // gradient accumulators of the parameters this thread owns: i = tid + 256 k
  constexpr int KOWN = (kMlpParams + kGradThreads - 1) / kGradThreads;
  float acc[KOWN];
#pragma unroll
  for (int k = 0; k < KOWN; ++k) acc[k] = 0.0f;
  float lsum = 0.0f;  // thread 0 only
  const int64_t begin = (int64_t)blockIdx.x * per_block;
  const int64_t end = begin + per_block < n ? begin + per_block : n;
  const float inv_n = 1.0f / (float)n;
  __syncthreads();
  for (int64_t s0 = begin; s0 < end; s0 += kSub) {
    const int nb = (int)(end - s0 < kSub ? end - s0 : kSub);
    for (int i = tid; i < kSub * kMlpIn; i += kGradThreads) {
      const int b = i / kMlpIn;
      xs[i] = b < nb ? bf16r(X[(s0 + b) * kMlpIn + (i - b * kMlpIn)]) : 0.0f;
    }
    __syncthreads();
    // layer 1
    for (int i = tid; i < kSub * 64; i += kGradThreads) {
      const int b = i >> 6, j = i & 63;
      float z = B1[j];
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) z = fmaf(W1[j * kMlpIn + k], xs[b * kMlpIn + k], z);
      float dg;
      a1[i] = gelu_acc(z, dg);
      z1[i] = dg;  // keep GELU'(z1) for the backward pass
    }
    __syncthreads();
    // layer 2
    for (int i = tid; i < kSub * 64; i += kGradThreads) {
      const int b = i >> 6, j = i & 63;
      float z = B2[j];
#pragma unroll 16
      for (int k = 0; k < 64; ++k) z = fmaf(W2[j * 64 + k], a1[b * 64 + k], z);
      float dg;
      a2[i] = gelu_acc(z, dg);
      z2[i] = dg;
    }
    __syncthreads();
    // outputs, loss (S5) and the output gradient
    if (tid < kSub) {
      const int b = tid;
      float o[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float z = B3[r];
        for (int k = 0; k < 64; ++k) z = fmaf(W3[r * 64 + k], a2[b * 64 + k], z);
        o[r] = z;
      }
      float l = 0.0f, d0 = 0.0f, d1 = 0.0f;
      if (b < nb) {
        const float yy = y[s0 + b];
        const float gh = sigm(o[0]);
        const float t = fabsf(gh - yy) < kTau ? 1.0f : 0.0f;
        l = (gh - yy) * (gh - yy) + kLam * (softplus(o[1]) - t * o[1]);
        d0 = 2.0f * (gh - yy) * gh * (1.0f - gh) * inv_n;
        d1 = kLam * (sigm(o[1]) - t) * inv_n;
      }
      dout[2 * b] = d0;
      dout[2 * b + 1] = d1;
      ls[b] = l;
    }
    __syncthreads();
    if (tid == 0)
      for (int b = 0; b < nb; ++b) lsum += ls[b];  // fixed order
    // dz2 = (dout W3) * GELU'(z2), in place of GELU'(z2)
    for (int i = tid; i < kSub * 64; i += kGradThreads) {
      const int b = i >> 6, j = i & 63;
      z2[i] *= fmaf(dout[2 * b], W3[j], dout[2 * b + 1] * W3[64 + j]);
    }
    __syncthreads();
    // dz1 = (dz2 W2) * GELU'(z1)
    for (int i = tid; i < kSub * 64; i += kGradThreads) {
      const int b = i >> 6, j = i & 63;
      float s = 0.0f;
#pragma unroll 16
      for (int k = 0; k < 64; ++k) s = fmaf(z2[b * 64 + k], W2[k * 64 + j], s);
      z1[i] *= s;
    }
    __syncthreads();
    // parameter gradients of this sub-batch, summed over its samples in order
#pragma unroll
    for (int k = 0; k < KOWN; ++k) {
      const int p = tid + kGradThreads * k;
      if (p >= kMlpParams) continue;
      float g = 0.0f;
      if (p < kMlpOffB1) {
        const int j = p / kMlpIn, c = p - j * kMlpIn;
        for (int b = 0; b < nb; ++b) g = fmaf(z1[b * 64 + j], xs[b * kMlpIn + c], g);
      } else if (p < kMlpOffW2) {
        const int j = p - kMlpOffB1;
        for (int b = 0; b < nb; ++b) g += z1[b * 64 + j];
      } else if (p < kMlpOffB2) {
        const int j = (p - kMlpOffW2) >> 6, c = (p - kMlpOffW2) & 63;
        for (int b = 0; b < nb; ++b) g = fmaf(z2[b * 64 + j], a1[b * 64 + c], g);
      } else if (p < kMlpOffW3) {
        const int j = p - kMlpOffB2;
        for (int b = 0; b < nb; ++b) g += z2[b * 64 + j];
      } else if (p < kMlpOffB3) {
        const int r = (p - kMlpOffW3) >> 6, c = (p - kMlpOffW3) & 63;
        for (int b = 0; b < nb; ++b) g = fmaf(dout[2 * b + r], a2[b * 64 + c], g);
      } else {
        const int r = p - kMlpOffB3;
        for (int b = 0; b < nb; ++b) g += dout[2 * b + r];
      }
      acc[k] += g;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < KOWN; ++k) {
    const int p = tid + kGradThreads * k;
    if (p < kMlpParams) gpart[(size_t)blockIdx.x * kMlpParams + p] = acc[k];
  }
  if (tid == 0) lpart[blockIdx.x] = lsum * inv_n;
}

// grad[p] = sum over blocks, in block order; loss likewise (block 0's thread 0).
__global__ void mlp_reduce_kernel(const float* __restrict__ gpart, const float* __restrict__ lpart, int nblk,
                                  float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += gpart[(size_t)b * kMlpParams + p];
    grad[p] = s;
  }
  if (p == 0) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += lpart[b];
    *loss = s;
  }
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t from the host).
__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ grad, float lr, float b1, float b2, float c1, float c2,
                                float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float g = grad[p];
  const float mm = fmaf(b1, m[p], (1.0f - b1) * g);
  const float vv = fmaf(b2, v[p], (1.0f - b2) * g * g);
  m[p] = mm;
  v[p] = vv;
  params[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace

namespace {

// FP32 master parameters -> tensor-core fragments (bf16, round to nearest even) + biases.
// Thread = (lane, slot) of one fragment.
__global__ void mlp_pack_kernel(const float* __restrict__ params, MlpPacked* __restrict__ out) {
  const float* W1 = params + kMlpOffW1;
  const float* W2 = params + kMlpOffW2;
  const float* W3 = params + kMlpOffW3;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = i & 31, g = lane >> 2, t = lane & 3, f = i >> 5;
  auto w1 = [&](int n, int k) { return k < kMlpIn ? W1[n * kMlpIn + k] : 0.0f; };
  auto w3 = [&](int n, int k) { return n < kMlpOut ? W3[n * 64 + k] : 0.0f; };
  if (f < 8) {  // layer 1, N tile f: B[k][n] = W1[n][k]
    const int n = 8 * f + g;
    out->w1[f][lane] = make_uint2(pack_bf16x2(w1(n, 2 * t), w1(n, 2 * t + 1)),
                                  pack_bf16x2(w1(n, 2 * t + 8), w1(n, 2 * t + 9)));
  } else if (f < 8 + 32) {  // layer 2, (kk, nt)
    const int kk = (f - 8) >> 3, nt = (f - 8) & 7, n = 8 * nt + g, k0 = 16 * kk + 2 * t;
    out->w2[kk][nt][lane] = make_uint2(pack_bf16x2(W2[n * 64 + k0], W2[n * 64 + k0 + 1]),
                                       pack_bf16x2(W2[n * 64 + k0 + 8], W2[n * 64 + k0 + 9]));
  } else if (f < 8 + 32 + 4) {  // layer 3, K step kk
    const int kk = f - 40, n = g, k0 = 16 * kk + 2 * t;
    out->w3[kk][lane] = make_uint2(pack_bf16x2(w3(n, k0), w3(n, k0 + 1)), pack_bf16x2(w3(n, k0 + 8), w3(n, k0 + 9)));
  } else if (f == 44) {
    out->b1[lane] = params[kMlpOffB1 + lane];
    out->b1[lane + 32] = params[kMlpOffB1 + lane + 32];
    out->b2[lane] = params[kMlpOffB2 + lane];
    out->b2[lane + 32] = params[kMlpOffB2 + lane + 32];
    if (lane < 4) out->b3[lane] = lane < kMlpOut ? params[kMlpOffB3 + lane] : 0.0f;
  }
}
constexpr int kPackThreads = 45 * 32;

// Stand-alone inference: one warp per 32 samples through the tensor-core routine of the
// fused stage kernel.  out[i][0] = o0, out[i][1] = o1 (pre-sigmoid outputs).
constexpr int kInferThreads = 128;
__global__ void __launch_bounds__(kInferThreads)
    mlp_infer_kernel(const MlpPacked* __restrict__ W, const float* __restrict__ X, int64_t n, float* __restrict__ out) {
  __shared__ __align__(16) MlpPacked sw;
  __shared__ __align__(16) __nv_bfloat16 xs[kInferThreads / 32][32 * 16];
  {
    const uint4* src = reinterpret_cast<const uint4*>(W);
    uint4* dst = reinterpret_cast<uint4*>(&sw);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpPacked) / 16); i += kInferThreads) dst[i] = src[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  for (int64_t base = ((int64_t)blockIdx.x * (kInferThreads / 32) + warp) * 32; base < n;
       base += (int64_t)gridDim.x * kInferThreads) {
    const int64_t i = base + (threadIdx.x & 31);
    float x[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = i < n ? X[i * kMlpIn + k] : 0.0f;
    float o0, o1;
    mlp_warp(sw, x, xs[warp], o0, o1);  // warp-uniform loop: every lane takes part
    if (i < n) {
      out[2 * i] = o0;
      out[2 * i + 1] = o1;
    }
  }
}

}  // namespace

struct cvweno_mlp_s {
  int device = 0;
  float* d_params = nullptr;  // FP32 master
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_grad = nullptr;
  float* d_loss = nullptr;
  float* d_gpart = nullptr;   // [kMaxGradBlocks][kMlpParams]
  float* d_lpart = nullptr;
  MlpPacked* d_packed = nullptr;
  unsigned int* d_fallbacks = nullptr;
  float* h_loss = nullptr;    // pinned
  int64_t step = 0;
};

namespace {

void free_mlp(cvweno_mlp n) {
  cudaFree(n->d_params);
  cudaFree(n->d_m);
  cudaFree(n->d_v);
  cudaFree(n->d_grad);
  cudaFree(n->d_loss);
  cudaFree(n->d_gpart);
  cudaFree(n->d_lpart);
  cudaFree(n->d_packed);
  cudaFree(n->d_fallbacks);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  delete n;
}

cudaError_t repack(cvweno_mlp n, cudaStream_t s) {
  mlp_pack_kernel<<<(kPackThreads + 127) / 128, 128, 0, s>>>(n->d_params, n->d_packed);
  return cudaGetLastError();
}

cudaError_t enqueue_grad(cvweno_mlp n, const float* X, const float* y, int64_t count, cudaStream_t s) {
  int64_t nblk = (count + kSub - 1) / kSub;
  if (nblk > kMaxGradBlocks) nblk = kMaxGradBlocks;
  const int64_t per_block = ((count + nblk - 1) / nblk + kSub - 1) / kSub * kSub;
  nblk = (count + per_block - 1) / per_block;
  const size_t smem = sizeof(float) * GradLayout::FLOATS;
  mlp_grad_kernel<<<(int)nblk, kGradThreads, smem, s>>>(n->d_params, X, y, count, per_block, n->d_gpart, n->d_lpart);
  mlp_reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(n->d_gpart, n->d_lpart, (int)nblk, n->d_grad,
                                                              n->d_loss);
  return cudaGetLastError();
}

cudaError_t enqueue_adam(cvweno_mlp n, float lr, cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999;
  n->step += 1;
  const float c1 = (float)(1.0 - pow(b1, (double)n->step)), c2 = (float)(1.0 - pow(b2, (double)n->step));
  mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(n->d_params, n->d_m, n->d_v, n->d_grad, lr, (float)b1,
                                                            (float)b2, c1, c2, 1e-8f);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

cvweno_status cvweno_mlp_create(const float* params, cvweno_mlp* out) {
  if (!out) return CVWENO_ERR_ARG;
  *out = nullptr;
  cvweno_mlp n = new (std::nothrow) cvweno_mlp_s;
  if (!n) return CVWENO_ERR_NOMEM;
  const size_t pb = sizeof(float) * kMlpParams;
  cudaError_t e = cudaGetDevice(&n->device);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_params, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_m, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_v, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_grad, pb);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->d_gpart, pb * kMaxGradBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_lpart, sizeof(float) * kMaxGradBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_packed, sizeof(MlpPacked));
  if (e == cudaSuccess) e = cudaMalloc(&n->d_fallbacks, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMallocHost(&n->h_loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->d_m, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(n->d_v, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(n->d_fallbacks, 0, sizeof(unsigned int));
  if (e == cudaSuccess)
    e = params ? cudaMemcpy(n->d_params, params, pb, cudaMemcpyHostToDevice) : cudaMemset(n->d_params, 0, pb);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * GradLayout::FLOATS));
  if (e == cudaSuccess) e = repack(n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_mlp(n);
    return CVWENO_ERR_CUDA;
  }
  *out = n;
  return CVWENO_OK;
}

cvweno_status cvweno_mlp_destroy(cvweno_mlp n) {
  if (!n) return CVWENO_ERR_ARG;
  cudaDeviceSynchronize();
  free_mlp(n);
  return CVWENO_OK;
}

cvweno_status cvweno_mlp_get_params(cvweno_mlp n, float* params) {
  if (!n || !params) return CVWENO_ERR_ARG;
  return cuda_status(cudaMemcpy(params, n->d_params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
}

cvweno_status cvweno_mlp_loss_grad(cvweno_mlp n, const float* X, const float* y, int64_t count, float* loss,
                                   float* grad, void* stream) {
  if (!n || !X || !y || count < 1) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  cudaError_t e = enqueue_grad(n, X, y, count, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(n->h_loss, n->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, n->d_grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && (loss || grad)) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  if (loss) *loss = *n->h_loss;
  return CVWENO_OK;
}

cvweno_status cvweno_mlp_adam_step(cvweno_mlp n, float lr, void* stream) {
  if (!n || !(lr > 0.0f)) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  cudaError_t e = enqueue_adam(n, lr, s);
  if (e == cudaSuccess) e = repack(n, s);
  return cuda_status(e);
}

cvweno_status cvweno_mlp_train(cvweno_mlp n, const float* X, const float* y, int64_t count, int64_t batch,
                               int epochs, float lr, float* last_loss, void* stream) {
  if (!n || !X || !y || count < 1 || batch < 1 || epochs < 0 || !(lr > 0.0f)) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  cudaError_t e = cudaSuccess;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep)
    for (int64_t b0 = 0; b0 < count && e == cudaSuccess; b0 += batch) {
      const int64_t nb = count - b0 < batch ? count - b0 : batch;
      e = enqueue_grad(n, X + b0 * kMlpIn, y + b0, nb, s);
      if (e == cudaSuccess) e = enqueue_adam(n, lr, s);
    }
  if (e == cudaSuccess) e = repack(n, s);
  if (e == cudaSuccess && last_loss)
    e = cudaMemcpyAsync(n->h_loss, n->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && last_loss) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  if (last_loss) *last_loss = epochs > 0 ? *n->h_loss : 0.0f;
  return CVWENO_OK;
}

cvweno_status cvweno_mlp_infer(cvweno_mlp n, const float* X, int64_t count, float* out, void* stream) {
  if (!n || !X || !out || count < 1) return CVWENO_ERR_ARG;
  const int64_t warps = (count + 31) / 32;
  int64_t blocks = (warps + kInferThreads / 32 - 1) / (kInferThreads / 32);
  if (blocks > 4 * 152) blocks = 4 * 152;
  mlp_infer_kernel<<<(int)blocks, kInferThreads, 0, S(stream)>>>(n->d_packed, X, count, out);
  return cuda_status(cudaGetLastError());
}

cvweno_status cvweno_features(cvweno_mesh m, const float* u, float* feats, float* gamma, float* norm,
                              void* stream) {
  if (!m || !u || !feats) return CVWENO_ERR_ARG;
  if (m->dim != 2 || m->kind != CVWENO_DG || m->desc.system == CVWENO_EULER) return CVWENO_ERR_UNSUPPORTED;
  StageArgs a = stage_base_args(m);
  a.u_in = u;
  a.feat_out = feats;
  a.gamma_out = gamma;
  a.norm_out = norm;
  a.mlp = nullptr;
  a.mode = kModeFeatures;
  return cuda_status(launch_stage(m, a, S(stream)));
}

cvweno_status cvweno_mesh_set_surrogate(cvweno_mesh m, cvweno_mlp n, float conf_min) {
  if (!m || !(conf_min >= 0.0f && conf_min <= 1.0f)) return CVWENO_ERR_ARG;
  if (n && (m->dim != 2 || m->kind != CVWENO_DG || m->desc.system == CVWENO_EULER)) return CVWENO_ERR_UNSUPPORTED;
  m->surrogate = n ? n->d_packed : nullptr;
  m->surrogate_conf_min = conf_min;
  m->surrogate_fallbacks = n ? n->d_fallbacks : nullptr;
  return CVWENO_OK;
}

cvweno_status cvweno_mlp_fallbacks(cvweno_mlp n, uint64_t* count, int reset, void* stream) {
  if (!n || !count) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  unsigned int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, n->d_fallbacks, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(n->d_fallbacks, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess && reset) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  *count = h;
  return CVWENO_OK;
}

}  // extern "C"
