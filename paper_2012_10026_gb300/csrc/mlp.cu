// Training and inference of the learned direction / binning controller: a
// 12-32-4 MLP with a ReLU hidden layer (no counterpart in the paper; it
// replaces the hand-tuned alpha/beta rule of Sec. 3.6 when selected).
//
//   forward     one warp per sample, lane j = hidden unit j, warp reductions
//               for the four outputs.
//   loss/grad   one block of MLP_WARPS warps; each warp accumulates the
//               gradient of its samples in registers (lane j owns row j of W1,
//               b1[j] and column j of W2), then the warps' partials are summed
//               in a fixed order in shared memory -- deterministic for a given
//               batch.
//   train       the same gradient inside a loop of full-batch Adam steps
//               (Kingma and Ba, 2015), parameters and moments in shared memory,
//               one launch for the whole run.
// Loss: L = 1/(2B) sum_b sum_k w_k (o_bk - y_bk)^2; ReLU'(0) = 0.
#include <math.h>
#include <string.h>

#include "g3_mlp.cuh"

#define MLP_WARPS 16
#define MLP_THREADS (MLP_WARPS * 32)
#define MLP_RED (MLP_NPARAMS + 1)  // gradient + loss per warp

// Accumulates the gradient of samples warp, warp + MLP_WARPS, ... into the
// warp's slot of red[] (MLP_RED floats per warp). P may live in shared or
// global memory.
__device__ void mlp_grad_partial(const float* P, const float* __restrict__ x,
                                 const float* __restrict__ y, const float* w4, int B,
                                 float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float invB = 1.f / (float)B;
  float gW1[MLP_IN], gb1 = 0.f, gW2[MLP_OUT], gb2[MLP_OUT], loss = 0.f;
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) gW1[i] = 0.f;
#pragma unroll
  for (int k = 0; k < MLP_OUT; ++k) gW2[k] = gb2[k] = 0.f;
  for (int s = warp; s < B; s += MLP_WARPS) {
    float f[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) f[i] = x[s * MLP_IN + i];
    float z = P[MLP_B1 + lane];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) z = fmaf(P[lane * MLP_IN + i], f[i], z);
    const float h = fmaxf(z, 0.f);
    float go[MLP_OUT];
#pragma unroll
    for (int k = 0; k < MLP_OUT; ++k) {
      float o = P[MLP_W2 + k * MLP_HID + lane] * h;
#pragma unroll
      for (int off = 16; off; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
      o += P[MLP_B2 + k];
      const float r = o - y[s * MLP_OUT + k];
      const float wk = w4 ? w4[k] : 1.f;
      go[k] = wk * r * invB;
      loss += 0.5f * wk * r * r * invB;
    }
    float gh = 0.f;
#pragma unroll
    for (int k = 0; k < MLP_OUT; ++k) {
      gW2[k] = fmaf(go[k], h, gW2[k]);
      gb2[k] += go[k];
      gh = fmaf(P[MLP_W2 + k * MLP_HID + lane], go[k], gh);
    }
    const float gz = z > 0.f ? gh : 0.f;
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) gW1[i] = fmaf(gz, f[i], gW1[i]);
    gb1 += gz;
  }
  float* r = red + warp * MLP_RED;
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) r[lane * MLP_IN + i] = gW1[i];
  r[MLP_B1 + lane] = gb1;
#pragma unroll
  for (int k = 0; k < MLP_OUT; ++k) r[MLP_W2 + k * MLP_HID + lane] = gW2[k];
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < MLP_OUT; ++k) r[MLP_B2 + k] = gb2[k];
    r[MLP_NPARAMS] = loss;
  }
}

// Sums the warps' partials in warp order: g[0..MLP_NPARAMS) and g[MLP_NPARAMS]
// = loss.
__device__ void mlp_grad_reduce(const float* red, float* g) {
  for (int p = threadIdx.x; p < MLP_RED; p += blockDim.x) {
    float s = 0.f;
    for (int wp = 0; wp < MLP_WARPS; ++wp) s += red[wp * MLP_RED + p];
    g[p] = s;
  }
}

__global__ void __launch_bounds__(MLP_THREADS) mlp_loss_grad_k(const float* P, const float* x,
                                                               const float* y, const float* w4,
                                                               int B, float* loss, float* grad) {
  __shared__ float red[MLP_WARPS * MLP_RED];
  __shared__ float g[MLP_RED];
  mlp_grad_partial(P, x, y, w4, B, red);
  __syncthreads();
  mlp_grad_reduce(red, g);
  __syncthreads();
  for (int p = threadIdx.x; p < MLP_NPARAMS; p += blockDim.x) grad[p] = g[p];
  if (threadIdx.x == 0) *loss = g[MLP_NPARAMS];
}

__global__ void __launch_bounds__(MLP_THREADS) mlp_train_k(float* params, const float* x,
                                                           const float* y, const float* w4,
                                                           int B, int steps, float lr,
                                                           float* losses) {
  __shared__ float red[MLP_WARPS * MLP_RED];
  __shared__ float g[MLP_RED];
  __shared__ float P[MLP_NPARAMS], m[MLP_NPARAMS], v[MLP_NPARAMS];
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int p = threadIdx.x; p < MLP_NPARAMS; p += blockDim.x) {
    P[p] = params[p];
    m[p] = 0.f;
    v[p] = 0.f;
  }
  __syncthreads();
  float b1t = 1.f, b2t = 1.f;
  for (int t = 1; t <= steps; ++t) {
    mlp_grad_partial(P, x, y, w4, B, red);
    __syncthreads();
    mlp_grad_reduce(red, g);
    __syncthreads();
    b1t *= b1;
    b2t *= b2;
    for (int p = threadIdx.x; p < MLP_NPARAMS; p += blockDim.x) {
      const float gp = g[p];
      m[p] = b1 * m[p] + (1.f - b1) * gp;
      v[p] = b2 * v[p] + (1.f - b2) * gp * gp;
      const float mh = m[p] / (1.f - b1t), vh = v[p] / (1.f - b2t);
      P[p] -= lr * mh / (sqrtf(vh) + eps);
    }
    if (threadIdx.x == 0 && losses) losses[t - 1] = g[MLP_NPARAMS];
    __syncthreads();
  }
  for (int p = threadIdx.x; p < MLP_NPARAMS; p += blockDim.x) params[p] = P[p];
}

__global__ void mlp_forward_k(const float* __restrict__ P, const float* __restrict__ x, int B,
                              float* out) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < B; s += nwarps) {
    float f[MLP_IN], o[MLP_OUT];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) f[i] = x[s * MLP_IN + i];
    mlp_eval_warp(P, f, o);
    if (lane == 0)
      for (int k = 0; k < MLP_OUT; ++k) out[s * MLP_OUT + k] = o[k];
  }
}

// Feature rows of logged levels, through the controller's own feature code.
struct FeatIn {
  long long nf, mf, nu, mu, prev_nf;
  int level, prev_dir;
};

__global__ void mlp_features_k(const FeatIn* in, int count, int32_t nb, int64_t nnz, float* x) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
    const FeatIn& r = in[s];
    mlp_features_raw(r.nf, r.mf, r.nu, r.mu, nb, nnz, r.prev_dir, r.level, r.prev_nf,
                     x + (size_t)s * MLP_IN);
  }
}

// ------------------------------------------------------------------ ABI
extern "C" g3_status g3_mlp_forward(const float* params, const float* x, int32_t B, float* out,
                                    void* stream) {
  if (!params || (B > 0 && (!x || !out)) || B < 0) {
    g3_set_error("g3_mlp_forward: bad arguments");
    return G3_EINVAL;
  }
  if (B == 0) return G3_OK;
  mlp_forward_k<<<g3_grid_for(B, 8), 256, 0, (cudaStream_t)stream>>>(params, x, B, out);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

extern "C" g3_status g3_mlp_loss_grad(const float* params, const float* x, const float* y,
                                      const float* w, int32_t B, float* loss, float* grad,
                                      void* stream) {
  if (!params || !x || !y || !loss || !grad || B <= 0) {
    g3_set_error("g3_mlp_loss_grad: bad arguments");
    return G3_EINVAL;
  }
  mlp_loss_grad_k<<<1, MLP_THREADS, 0, (cudaStream_t)stream>>>(params, x, y, w, B, loss, grad);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

extern "C" g3_status g3_mlp_train(float* params, const float* x, const float* y, const float* w,
                                  int32_t B, int32_t steps, float lr, float* losses,
                                  void* stream) {
  if (!params || !x || !y || B <= 0 || steps < 0 || !(lr > 0.f)) {
    g3_set_error("g3_mlp_train: bad arguments");
    return G3_EINVAL;
  }
  if (steps == 0) return G3_OK;
  mlp_train_k<<<1, MLP_THREADS, 0, (cudaStream_t)stream>>>(params, x, y, w, B, steps, lr,
                                                           losses);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

extern "C" g3_status g3_mlp_features(const g3_level_stats* stats, int32_t count, int32_t n_bfs,
                                     int64_t nnz, float* x, void* stream) {
  if (count < 0 || nnz < 0 || (count > 0 && (!stats || !x))) {
    g3_set_error("g3_mlp_features: bad arguments");
    return G3_EINVAL;
  }
  if (count == 0) return G3_OK;
  cudaStream_t s = (cudaStream_t)stream;
  FeatIn* h = (FeatIn*)malloc(sizeof(FeatIn) * (size_t)count);
  if (!h) return G3_ENOMEM;
  for (int i = 0; i < count; ++i) {
    const g3_level_stats& r = stats[i];
    h[i].nf = r.n_f;
    h[i].mf = r.m_f;
    h[i].nu = r.n_u;
    h[i].mu = r.m_u;
    h[i].level = r.level;
    // the previous level of the same search is the preceding record
    h[i].prev_dir = (r.level > 0 && i > 0) ? stats[i - 1].dir : 0;
    h[i].prev_nf = (r.level > 0 && i > 0) ? stats[i - 1].n_f : 0;
  }
  FeatIn* d = nullptr;
  g3_status st = g3_alloc(&d, (size_t)count, s);
  if (st == G3_OK) {
    cudaError_t e = cudaMemcpyAsync(d, h, sizeof(FeatIn) * (size_t)count,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      mlp_features_k<<<g3_grid_for(count, 256), 256, 0, s>>>(d, count, n_bfs, nnz, x);
      g3_count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // h is read by the copy
    if (e != cudaSuccess) {
      g3_set_error("g3_mlp_features: %s", cudaGetErrorString(e));
      st = G3_ECUDA;
    }
    g3_free(d, s);
  }
  free(h);
  return st;
}
