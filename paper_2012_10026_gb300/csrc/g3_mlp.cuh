// The 12-32-4 MLP of the learned direction / binning controller: feature
// extraction and one-warp inference, shared by the controller kernel (bfs.cu)
// and the training kernels (mlp.cu) so training sees exactly the features the
// controller computes.
#pragma once
#include "g3_internal.cuh"

#define MLP_IN 12
#define MLP_HID 32
#define MLP_OUT 4
#define MLP_NPARAMS (MLP_HID * MLP_IN + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT)  // 548
// parameter layout: W1[32][12], b1[32], W2[4][32], b2[4]
#define MLP_B1 (MLP_HID * MLP_IN)
#define MLP_W2 (MLP_B1 + MLP_HID)
#define MLP_B2 (MLP_W2 + MLP_OUT * MLP_HID)

// Features of the frontier F_L (see the controller's documentation), all
// from the frontier sizes and degree sums the expansion kernels count anyway
// (n: vertices of the searched graph, nnz: its directed entries):
//  0 log2((1+n_f)/(1+n))   1 log2((1+m_f)/(1+nnz))
//  2 log2((1+n_u)/(1+n))   3 n / 2^24: the graph size, linear, because a
//    bottom-up step's walk over the bitmap costs time in proportion to n
//    while a small top-down step's cost does not grow with it
//  4 log2((1+m_f)/(1+n_f)) / 16: mean degree of the frontier
//  5 log2((1+m_f)/(1+m_u))
//  6 log2((1+n)/(32 (1+m_f))): bitmap words a bottom-up step walks per
//    frontier edge a top-down step expands   7 previous direction
//  8 log2((1+m_u)/(1+n_u)) / 16: mean degree of the unvisited vertices
//  9 log2((1+n_f)/(1+n_f of the previous level)) / 8: frontier growth
// 10 min(level, 32) / 32    11 1 - n_u / n: fraction of the graph visited
__device__ __forceinline__ void mlp_features_raw(long long nf, long long mf, long long nu,
                                                 long long mu, int32_t nb, long long nnz,
                                                 int prev_dir, int level, long long prev_nf,
                                                 float* f) {
  const float fnf = (float)nf, fmf = (float)mf, fnu = (float)nu, fmu = (float)mu;
  const float fn = (float)nb, fe = (float)nnz;
  f[0] = log2f((1.f + fnf) / (1.f + fn));
  f[1] = log2f((1.f + fmf) / (1.f + fe));
  f[2] = log2f((1.f + fnu) / (1.f + fn));
  f[3] = fn * (1.f / 16777216.f);
  f[4] = log2f((1.f + fmf) / (1.f + fnf)) * (1.f / 16.f);
  f[5] = log2f((1.f + fmf) / (1.f + fmu));
  f[6] = log2f((1.f + fn) / (32.f * (1.f + fmf)));
  f[7] = (float)prev_dir;
  f[8] = log2f((1.f + fmu) / (1.f + fnu)) * (1.f / 16.f);
  f[9] = log2f((1.f + fnf) / (1.f + (float)prev_nf)) * (1.f / 8.f);
  f[10] = (float)(level < 32 ? level : 32) * (1.f / 32.f);
  f[11] = nb > 0 ? 1.f - fnu / fn : 0.f;
}

// One lane's share of the weights: hidden unit j's input row and bias, and
// its weight into each output. Loaded before the features are known, so that
// their latency overlaps the work that produces the features.
struct MlpLane {
  float w1[MLP_IN], b1, w2[MLP_OUT], b2[MLP_OUT];
};

__device__ __forceinline__ void mlp_load_lane(const float* __restrict__ P, MlpLane& L) {
  const int j = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) L.w1[i] = P[j * MLP_IN + i];
  L.b1 = P[MLP_B1 + j];
#pragma unroll
  for (int k = 0; k < MLP_OUT; ++k) {
    L.w2[k] = P[MLP_W2 + k * MLP_HID + j];
    L.b2[k] = P[MLP_B2 + k];
  }
}

// One warp evaluates the network for one feature vector: lane j is hidden
// unit j; the four outputs are warp reductions.
__device__ __forceinline__ void mlp_eval_lane(const MlpLane& L, const float* f, float* out) {
  float z = L.b1;
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) z = fmaf(L.w1[i], f[i], z);
  const float h = fmaxf(z, 0.f);
#pragma unroll
  for (int k = 0; k < MLP_OUT; ++k) {
    float s = L.w2[k] * h;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    out[k] = s + L.b2[k];
  }
}

__device__ __forceinline__ void mlp_eval_warp(const float* __restrict__ P, const float* f,
                                              float* out) {
  MlpLane L;
  mlp_load_lane(P, L);
  mlp_eval_lane(L, f, out);
}
