/*
 * Host (C, OpenMP) generator of the seeded synthetic inputs; the CUDA twin in
 * gg_dev.cu produces the same bytes. Inputs only: no part of the method.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "gg_common.h"

static int gg_bits_for(int64_t n) {
  int b = 0;
  while ((1LL << b) < n) ++b;
  return b < 1 ? 1 : b;
}

/* Kronecker edges [e0, e0+count) of a graph with 2^scale vertices. */
void gg_kron(uint64_t seed, int scale, int64_t e0, int64_t count, uint32_t tA,
             uint32_t tAB, uint32_t tABC, int32_t* src, int32_t* dst) {
  const uint64_t ke = gg_key(seed, GG_EDGES), kp = gg_key(seed, GG_PERM);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i)
    gg_kron_edge(ke, kp, scale, tA, tAB, tABC, (uint64_t)(e0 + i), &src[i], &dst[i]);
}

/* Chung-Lu edges [e0, e0+count) over n vertices with cumulative table cum. */
void gg_chunglu(uint64_t seed, int64_t n, const uint64_t* cum, int64_t e0,
                int64_t count, int32_t* src, int32_t* dst) {
  const uint64_t ke = gg_key(seed, GG_EDGES), kp = gg_key(seed, GG_PERM);
  const int bits = gg_bits_for(n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i)
    gg_chunglu_edge(ke, kp, bits, n, cum, (uint64_t)(e0 + i), &src[i], &dst[i]);
}

/* flags[v] = 1 when v has an incident edge with distinct endpoints. */
void gg_mark_nonisolated(const int32_t* src, const int32_t* dst, int64_t m,
                         int32_t n, uint8_t* flags) {
  memset(flags, 0, (size_t)n);
  for (int64_t i = 0; i < m; ++i)
    if (src[i] != dst[i]) { flags[src[i]] = 1; flags[dst[i]] = 1; }
}

/* Up to k distinct roots drawn uniformly among vertices with flags[v] != 0,
 * in draw order. Returns how many were found (fewer when the graph has
 * fewer than k candidates). */
int32_t gg_pick_roots(const uint8_t* flags, int32_t n, int32_t k, uint64_t seed,
                      int32_t* out) {
  const uint64_t kr = gg_key(seed, GG_ROOTS);
  int64_t cand = 0;
  for (int32_t v = 0; v < n; ++v) cand += flags[v] != 0;
  if (cand < k) k = (int32_t)cand;
  uint8_t* taken = (uint8_t*)calloc((size_t)n > 0 ? (size_t)n : 1, 1);
  int32_t got = 0;
  for (uint64_t i = 0; got < k; ++i) {
    int32_t v = (int32_t)(gg_draw(kr, i) % (uint64_t)n);
    if (flags[v] && !taken[v]) { taken[v] = 1; out[got++] = v; }
  }
  free(taken);
  return got;
}

/* Image of x under the seeded bijection on [0, n) (exposed for tests). */
int64_t gg_perm_value(uint64_t seed, int64_t n, int64_t x) {
  return (int64_t)gg_perm((uint64_t)x, gg_key(seed, GG_PERM), gg_bits_for(n), (uint64_t)n);
}

/* Raw draw (exposed for tests). */
uint64_t gg_draw_value(uint64_t seed, uint64_t purpose, uint64_t ctr) {
  return gg_draw(gg_key(seed, purpose), ctr);
}
