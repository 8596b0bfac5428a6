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
// (n: vertices of the searched graph, nnz: its directed entries), and all
// ratios of the graph's own counts, so that a level looks the same to the
// network on a graph of any size:
//  0 log2((1+n_f)/(1+n))   1 log2((1+m_f)/(1+nnz))
//  2 log2((1+n_u)/(1+n))   3 log2((1+n_u)/(1+n_f)) / 8: unvisited vertices per
//    frontier vertex
//  4 log2((1+m_f)/(1+n_f)) / 16: mean degree of the frontier
//  5 log2((1+m_f)/(1+m_u))
//  6 log2((1+n)/(32 (1+m_f))): bitmap words a bottom-up step walks per
//    frontier edge a top-down step expands   7 previous direction
//  8 log2((1+m_u)/(1+n_u)) / 16: mean degree of the unvisited vertices
//  9 log2((1+n_f)/(1+n_f of the previous level)) / 8: frontier growth
// 10 min(level, 32) / 32    11 1 - n_u / n: fraction of the graph visited
// Feature j alone, so that the lanes of a warp can compute them at once.
// Nine of them are log2((1+a)/(1+b)) * scale + shift for a pair of counts;
// the pair is selected per lane and every lane runs the same instructions
// (one log2f per lane instead of the warp stepping through twelve cases).
__device__ __forceinline__ float mlp_feature(int j, long long nf, long long mf, long long nu,
                                             long long mu, int32_t nb, long long nnz,
                                             int prev_dir, int level, long long prev_nf) {
  const float fnf = (float)nf, fmf = (float)mf, fnu = (float)nu, fmu = (float)mu;
  const float fn = (float)nb, fe = (float)nnz, fpn = (float)prev_nf;
  // numerator and denominator counts of the log features
  const float a = j == 0 ? fnf : j == 1 ? fmf : j == 2 ? fnu : j == 3 ? fnu : j == 4 ? fmf
                : j == 5 ? fmf : j == 6 ? fn : j == 8 ? fmu : fnf;
  const float b = j == 0 ? fn : j == 1 ? fe : j == 2 ? fn : j == 3 ? fnf : j == 4 ? fnf
                : j == 5 ? fmu : j == 6 ? fmf : j == 8 ? fnu : fpn;
  const float scale = j == 3 || j == 9 ? 1.f / 8.f : (j == 4 || j == 8 ? 1.f / 16.f : 1.f);
  const float shift = j == 6 ? -5.f : 0.f;  // 6: per 32 (1 + m_f), a word per 32 vertices
  const float lg = log2f((1.f + a) / (1.f + b)) * scale + shift;
  const float lv = (float)(level < 32 ? level : 32) * (1.f / 32.f);
  const float vis = nb > 0 ? 1.f - fnu / fn : 0.f;
  return j == 7 ? (float)prev_dir : j == 10 ? lv : j == 11 ? vis : lg;
}

__device__ __forceinline__ void mlp_features_raw(long long nf, long long mf, long long nu,
                                                 long long mu, int32_t nb, long long nnz,
                                                 int prev_dir, int level, long long prev_nf,
                                                 float* f) {
#pragma unroll
  for (int j = 0; j < MLP_IN; ++j)
    f[j] = mlp_feature(j, nf, mf, nu, mu, nb, nnz, prev_dir, level, prev_nf);
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
