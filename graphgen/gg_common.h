/*
 * Seeded, counter-based synthetic graph generators (inputs only).
 *
 * This header holds the definitions shared by the host generator (gg_host.c)
 * and its CUDA twin (gg_dev.cu): both compile exactly these integer
 * functions, so the two produce bit-identical edge lists for the same seed.
 * Nothing here computes any part of the BFS/RCM method; the generators stand
 * in for the Graph500 Kronecker generator of the paper's evaluation (Sec. 4.2)
 * and for a Chung-Lu power-law graph.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used in counter mode: draw i
 * of stream `key` is the SplitMix64 output function applied to
 * key + (i + 1) * golden_gamma.  Every draw is independent of every other,
 * so generation is embarrassingly parallel and order-free.
 */
#ifndef GG_COMMON_H
#define GG_COMMON_H
#include <stdint.h>

#if defined(__CUDACC__)
#define GG_HD static __host__ __device__ __forceinline__
#else
#define GG_HD static inline
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

/* SplitMix64 output ("mix") function. */
GG_HD uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Stream key for (seed, purpose): purposes keep edge draws, the vertex
 * relabelling and root choice independent of one another. */
GG_HD uint64_t gg_key(uint64_t seed, uint64_t purpose) {
  return gg_mix64(seed * 0x100ULL + purpose + 0x632BE59BD9B4E019ULL);
}

/* Draw number `ctr` of stream `key` (counter mode). */
GG_HD uint64_t gg_draw(uint64_t key, uint64_t ctr) {
  return gg_mix64(key + (ctr + 1ULL) * GG_GAMMA);
}

enum { GG_EDGES = 1, GG_PERM = 2, GG_ROOTS = 3, GG_SCALE = 4 };

/* Seeded bijection on [0, 2^bits): four rounds of an odd multiply-add modulo
 * 2^bits followed by an xorshift, each step invertible on bits-bit words. */
GG_HD uint64_t gg_perm_pow2(uint64_t x, uint64_t kperm, int bits) {
  const uint64_t mask = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1ULL);
  const int sh = (bits + 1) / 2;
  for (int r = 0; r < 4; ++r) {
    uint64_t mul = (gg_draw(kperm, 2 * r) | 1ULL) & mask;
    uint64_t add = gg_draw(kperm, 2 * r + 1) & mask;
    x = (x * mul + add) & mask;
    x ^= x >> sh;
  }
  return x;
}

/* Bijection on [0, n) by cycle-walking the power-of-two bijection. */
GG_HD uint64_t gg_perm(uint64_t x, uint64_t kperm, int bits, uint64_t n) {
  do {
    x = gg_perm_pow2(x, kperm, bits);
  } while (x >= n);
  return x;
}

/* Kronecker (R-MAT) edge e at the given scale: one draw per bit level picks
 * a quadrant of the 2x2 initiator, compared as 32-bit integers against the
 * cumulative thresholds tA <= tAB <= tABC (probabilities times 2^32). The
 * endpoints are then relabelled by the seeded bijection. */
GG_HD void gg_kron_edge(uint64_t kedge, uint64_t kperm, int scale, uint32_t tA,
                        uint32_t tAB, uint32_t tABC, uint64_t e, int32_t* u_out,
                        int32_t* v_out) {
  uint64_t u = 0, v = 0;
  for (int l = 0; l < scale; ++l) {
    uint32_t r = (uint32_t)(gg_draw(kedge, e * (uint64_t)scale + (uint64_t)l) >> 32);
    uint64_t bu, bv;
    if (r < tA) {
      bu = 0; bv = 0;
    } else if (r < tAB) {
      bu = 0; bv = 1;
    } else if (r < tABC) {
      bu = 1; bv = 0;
    } else {
      bu = 1; bv = 1;
    }
    u |= bu << l;
    v |= bv << l;
  }
  *u_out = (int32_t)gg_perm_pow2(u, kperm, scale);
  *v_out = (int32_t)gg_perm_pow2(v, kperm, scale);
}

/* First index i in [0, n) with r < cum[i]; n-1 when none (r == 2^64-1). */
GG_HD int64_t gg_upper_bound(const uint64_t* cum, int64_t n, uint64_t r) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (r < cum[mid]) hi = mid; else lo = mid + 1;
  }
  return lo < n ? lo : n - 1;
}

/* Chung-Lu edge e: both endpoints drawn with probability proportional to the
 * weight table (given as an integer cumulative table), then relabelled. */
GG_HD void gg_chunglu_edge(uint64_t kedge, uint64_t kperm, int bits, int64_t n,
                           const uint64_t* cum, uint64_t e, int32_t* u_out,
                           int32_t* v_out) {
  int64_t u = gg_upper_bound(cum, n, gg_draw(kedge, 2 * e));
  int64_t v = gg_upper_bound(cum, n, gg_draw(kedge, 2 * e + 1));
  *u_out = (int32_t)gg_perm((uint64_t)u, kperm, bits, (uint64_t)n);
  *v_out = (int32_t)gg_perm((uint64_t)v, kperm, bits, (uint64_t)n);
}

#endif /* GG_COMMON_H */
