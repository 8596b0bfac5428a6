/*
 * CUDA twin of the host generator (gg_host.c): the same integer functions
 * from gg_common.h, one thread per edge, so both produce identical bytes.
 * Inputs only: no part of the method.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include "gg_common.h"

static int gg_bits_for(int64_t n) {
  int b = 0;
  while ((1LL << b) < n) ++b;
  return b < 1 ? 1 : b;
}

__global__ void gg_kron_kernel(uint64_t ke, uint64_t kp, int scale, uint32_t tA,
                               uint32_t tAB, uint32_t tABC, int64_t e0,
                               int64_t count, int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    gg_kron_edge(ke, kp, scale, tA, tAB, tABC, (uint64_t)(e0 + i), &src[i], &dst[i]);
}

__global__ void gg_chunglu_kernel(uint64_t ke, uint64_t kp, int bits, int64_t n,
                                  const uint64_t* cum, int64_t e0, int64_t count,
                                  int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    gg_chunglu_edge(ke, kp, bits, n, cum, (uint64_t)(e0 + i), &src[i], &dst[i]);
}

__global__ void gg_mark_kernel(const int32_t* src, const int32_t* dst, int64_t m,
                               uint8_t* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[i], v = dst[i];
    if (u != v) { flags[u] = 1; flags[v] = 1; }
  }
}

static int gg_grid(int64_t count) {
  int64_t b = (count + 255) / 256;
  if (b > 152 * 64) b = 152 * 64;
  return b < 1 ? 1 : (int)b;
}

extern "C" int gg_kron_dev(uint64_t seed, int scale, int64_t e0, int64_t count,
                           uint32_t tA, uint32_t tAB, uint32_t tABC, int32_t* src,
                           int32_t* dst, void* stream) {
  if (count <= 0) return 0;
  gg_kron_kernel<<<gg_grid(count), 256, 0, (cudaStream_t)stream>>>(
      gg_key(seed, GG_EDGES), gg_key(seed, GG_PERM), scale, tA, tAB, tABC, e0,
      count, src, dst);
  return (int)cudaGetLastError();
}

extern "C" int gg_chunglu_dev(uint64_t seed, int64_t n, const uint64_t* cum,
                              int64_t e0, int64_t count, int32_t* src,
                              int32_t* dst, void* stream) {
  if (count <= 0) return 0;
  gg_chunglu_kernel<<<gg_grid(count), 256, 0, (cudaStream_t)stream>>>(
      gg_key(seed, GG_EDGES), gg_key(seed, GG_PERM), gg_bits_for(n), n, cum, e0,
      count, src, dst);
  return (int)cudaGetLastError();
}

/* flags must hold n zeroed bytes. */
extern "C" int gg_mark_nonisolated_dev(const int32_t* src, const int32_t* dst,
                                       int64_t m, uint8_t* flags, void* stream) {
  if (m <= 0) return 0;
  gg_mark_kernel<<<gg_grid(m), 256, 0, (cudaStream_t)stream>>>(src, dst, m, flags);
  return (int)cudaGetLastError();
}
