/*
 * Multithreaded hybrid BFS on the host cores: the paper's own CPU design
 * (Jiang et al., PPoPP'21, Sec. 3.3-3.5), kept as a second CPU baseline
 * beside the serial oracle. It is not part of the GPU library and the GPU
 * path never calls it.
 *
 * What it follows:
 *   - top-down, phase 1 (before the first bottom-up step): Algorithm 4. Every
 *     thread walks the whole frontier; thread i takes the i-th of t equal
 *     blocks of each frontier vertex's neighbour list (Eq. 3: workload =
 *     degree / t, startpos_k = row start + k * workload), and the remainder
 *     past startpos_t goes to thread (j mod t) for the j-th frontier vertex.
 *     A neighbour is claimed by an atomic test-and-set of its visited bit.
 *   - top-down, phase 3 (after a bottom-up step): Algorithm 1, frontier
 *     vertices statically divided among the threads.
 *   - bottom-up: Algorithm 6 (Algorithm 5's partitions plus the two
 *     workload reductions). The bitmap is cut into lambda * t partitions of
 *     whole 64-byte blocks whose sizes form a descending arithmetic sequence
 *     (degrees ascend with the RCM label, Sec. 3.4); threads take the next
 *     partition with fetch_add. Each partition is first shrunk past its
 *     all-visited words at both ends (kept across steps), then every
 *     unvisited vertex probes its highest-degree neighbour (neighbors+), then
 *     the partition is shrunk again and the rest scan the remaining
 *     neighbours in decreasing degree (neighbors-). Under RCM a higher label
 *     means a higher degree (Sec. 3.4), so neighbors+ is the row's last entry
 *     and neighbors- the row read backwards (the same reading as the GPU
 *     path's degree-aware scan).
 *   - SIMD (Sec. 3.5): next-frontier words are ORed into visited 128 bits at
 *     a time after each bottom-up loop, and thread-local queue buffers are
 *     copied into the shared queue 128 bits at a time; NEON intrinsics where
 *     the compiler targets ARM (vld1q_u64 / vst1q_u64 / vorrq_u64), the same
 *     operations on two 64-bit words elsewhere.
 *   - direction: after a top-down level go bottom-up when m_f * alpha > m_u;
 *     after a bottom-up level return top-down when the frontier shrank and
 *     n_f * beta < n (Sec. 2.1 / Sec. 3.6; the rule the GPU path uses).
 *
 * The graph is the RCM-relabelled CSR over the n' non-isolated vertices, rows
 * ascending; outputs are parent[] and level[] in original IDs, -1 where
 * unreached, as the GPU library returns them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#if defined(__ARM_NEON)
#include <arm_neon.h>
#endif

#define HB_BLOCK_WORDS 8 /* 64-byte cache-line block of the bitmaps */
#define HB_LOCAL 4096    /* thread-local queue buffer entries */

typedef struct {
  int32_t alpha, beta; /* direction rule (14, 24) */
  int32_t lambda;      /* partitions per thread (20, Sec. 3.4 / Fig. 4) */
  int32_t threads;     /* 0: omp_get_max_threads() */
  int32_t td_kind;     /* 0: Algorithm 4 before the first bottom-up step,
                          Algorithm 1 after it; 1: always Algorithm 4;
                          2: always Algorithm 1 */
  int32_t reserved[3];
} hb_opts;

typedef struct {
  int32_t levels, bu_levels, td_levels, threads;
  int64_t bu_examined; /* edges examined by bottom-up steps */
} hb_stats;

struct hb_ws {
  int32_t nb, n, t;
  int64_t words;        /* 64-bit bitmap words, padded to whole blocks */
  int64_t blocks;       /* 64-byte blocks */
  const int64_t* off;
  const int32_t* col;
  const int32_t* old_of_new;
  const int32_t* new_of_old;
  uint64_t *visited, *fa, *fb;
  int32_t *pi, *lev, *qa, *qb;
  int64_t nparts, *part_lo, *part_hi; /* word ranges, shrunk across steps */
  int64_t* part_base;                 /* initial ranges */
};

typedef struct hb_ws hb_ws;

/* ------------------------------------------------------------- SIMD */

static void copy_128(int32_t* dst, const int32_t* src, int64_t count) {
  int64_t i = 0;
#if defined(__ARM_NEON)
  for (; i + 4 <= count; i += 4) vst1q_s32(dst + i, vld1q_s32(src + i));
#else
  for (; i + 4 <= count; i += 4) {
    uint64_t a, b;
    memcpy(&a, src + i, 8);
    memcpy(&b, src + i + 2, 8);
    memcpy(dst + i, &a, 8);
    memcpy(dst + i + 2, &b, 8);
  }
#endif
  for (; i < count; ++i) dst[i] = src[i];
}

/* visited[w] |= next[w] over [w0, w1), 128 bits at a time */
static void or_128(uint64_t* visited, const uint64_t* next, int64_t w0, int64_t w1) {
  int64_t w = w0;
#if defined(__ARM_NEON)
  for (; w + 2 <= w1; w += 2)
    vst1q_u64(visited + w, vorrq_u64(vld1q_u64(visited + w), vld1q_u64(next + w)));
#else
  for (; w + 2 <= w1; w += 2) {
    visited[w] |= next[w];
    visited[w + 1] |= next[w + 1];
  }
#endif
  for (; w < w1; ++w) visited[w] |= next[w];
}

/* ------------------------------------------------------- workspace */

void hb_ws_free(hb_ws* ws) {
  if (!ws) return;
  free(ws->visited);
  free(ws->fa);
  free(ws->fb);
  free(ws->pi);
  free(ws->lev);
  free(ws->qa);
  free(ws->qb);
  free(ws->part_lo);
  free(ws->part_hi);
  free(ws->part_base);
  free(ws);
}

static void* alloc64(size_t bytes) {
  void* p = NULL;
  if (posix_memalign(&p, 64, bytes ? bytes : 64) != 0) return NULL;
  return p;
}

/* Partition boundaries in blocks: nparts partitions whose sizes follow the
 * weights nparts, nparts - 1, ..., 1 (a descending arithmetic sequence),
 * boundaries rounded down so that they ascend and cover [0, blocks).
 * bound[k] for k = 0..nparts. */
void hb_partitions(int64_t blocks, int64_t nparts, int64_t* bound) {
  const double total = (double)nparts * (double)(nparts + 1) / 2.0;
  double acc = 0.0;
  bound[0] = 0;
  for (int64_t k = 0; k < nparts; ++k) {
    acc += (double)(nparts - k);
    int64_t b = (int64_t)((double)blocks * (acc / total));
    if (k == nparts - 1) b = blocks;
    if (b < bound[k]) b = bound[k];
    bound[k + 1] = b;
  }
}

/* Workspace for one graph: the RCM CSR over nb vertices (off: nb+1, col),
 * the permutation (old_of_new, new_of_old: n entries each; NULL for an
 * unrelabelled graph with nb == n). The arrays are borrowed, not copied.
 * lambda and threads fix the partitions. Returns NULL when out of memory. */
hb_ws* hb_ws_create(const int64_t* off, const int32_t* col, int32_t nb,
                    const int32_t* old_of_new, const int32_t* new_of_old, int32_t n,
                    int32_t lambda, int32_t threads) {
  hb_ws* ws = (hb_ws*)calloc(1, sizeof(hb_ws));
  if (!ws) return NULL;
  ws->nb = nb;
  ws->n = n;
  ws->t = threads > 0 ? threads : omp_get_max_threads();
  ws->off = off;
  ws->col = col;
  ws->old_of_new = old_of_new;
  ws->new_of_old = new_of_old;
  ws->blocks = ((int64_t)nb + 511) / 512;
  ws->words = ws->blocks * HB_BLOCK_WORDS;
  const size_t wb = (size_t)ws->words * 8, vb = ((size_t)nb + 1) * 4;
  ws->visited = (uint64_t*)alloc64(wb);
  ws->fa = (uint64_t*)alloc64(wb);
  ws->fb = (uint64_t*)alloc64(wb);
  ws->pi = (int32_t*)alloc64(vb);
  ws->lev = (int32_t*)alloc64(vb);
  ws->qa = (int32_t*)alloc64(vb);
  ws->qb = (int32_t*)alloc64(vb);
  int64_t np = (int64_t)(lambda > 0 ? lambda : 20) * ws->t;
  if (np > ws->blocks) np = ws->blocks > 0 ? ws->blocks : 1;
  ws->nparts = np;
  ws->part_lo = (int64_t*)calloc((size_t)np + 1, 8);
  ws->part_hi = (int64_t*)calloc((size_t)np + 1, 8);
  ws->part_base = (int64_t*)calloc((size_t)np + 1, 8);
  if (!ws->visited || !ws->fa || !ws->fb || !ws->pi || !ws->lev || !ws->qa || !ws->qb ||
      !ws->part_lo || !ws->part_hi || !ws->part_base) {
    hb_ws_free(ws);
    return NULL;
  }
  hb_partitions(ws->blocks, np, ws->part_base);
  return ws;
}

/* ------------------------------------------------------------ steps */

static inline int bit_of(const uint64_t* bm, int32_t v) { return (bm[v >> 6] >> (v & 63)) & 1u; }

/* atomic test-and-set of v's visited bit; 1 when this call set it */
static inline int claim(uint64_t* visited, int32_t v) {
  const uint64_t m = 1ull << (v & 63);
  if (__atomic_load_n(&visited[v >> 6], __ATOMIC_RELAXED) & m) return 0;
  return !(__atomic_fetch_or(&visited[v >> 6], m, __ATOMIC_RELAXED) & m);
}

typedef struct {
  int32_t buf[HB_LOCAL];
  int32_t cnt;
  int64_t mf; /* degree sum of what this thread discovered */
} local_q;

static void lq_flush(local_q* lq, int32_t* gq, int64_t* glen) {
  if (!lq->cnt) return;
  const int64_t base = __atomic_fetch_add(glen, (int64_t)lq->cnt, __ATOMIC_RELAXED);
  copy_128(gq + base, lq->buf, lq->cnt);
  lq->cnt = 0;
}

static inline void visit(hb_ws* ws, local_q* lq, int32_t* gq, int64_t* glen, int32_t w,
                         int32_t v, int32_t L1) {
  if (!claim(ws->visited, w)) return;
  ws->pi[w] = v;
  ws->lev[w] = L1;
  lq->mf += ws->off[w + 1] - ws->off[w];
  lq->buf[lq->cnt++] = w;
  if (lq->cnt == HB_LOCAL) lq_flush(lq, gq, glen);
}

/* Algorithm 4 (td_kind 1) or Algorithm 1 (td_kind 2): queue cur -> queue
 * next; returns |F_next|, *mf its degree sum. */
static int64_t top_down(hb_ws* ws, const int32_t* cur, int64_t nf, int32_t* next,
                        int32_t L1, int alg4, int64_t* mf) {
  int64_t len = 0, msum = 0;
  const int t = ws->t;
#pragma omp parallel num_threads(t) reduction(+ : msum)
  {
    local_q* lq = (local_q*)malloc(sizeof(local_q));
    lq->cnt = 0;
    lq->mf = 0;
    const int i = omp_get_thread_num(), nt = omp_get_num_threads();
    if (alg4) {
      for (int64_t j = 0; j < nf; ++j) {
        const int32_t v = cur[j];
        const int64_t b = ws->off[v], e = ws->off[v + 1];
        const int64_t workload = (e - b) / nt;
        const int64_t s0 = b + (int64_t)i * workload;
        for (int64_t k = s0; k < s0 + workload; ++k) visit(ws, lq, next, &len, ws->col[k], v, L1);
        if (i == (int)(j % nt))
          for (int64_t k = b + (int64_t)nt * workload; k < e; ++k)
            visit(ws, lq, next, &len, ws->col[k], v, L1);
      }
    } else {
#pragma omp for schedule(static)
      for (int64_t j = 0; j < nf; ++j) {
        const int32_t v = cur[j];
        for (int64_t k = ws->off[v]; k < ws->off[v + 1]; ++k)
          visit(ws, lq, next, &len, ws->col[k], v, L1);
      }
    }
    lq_flush(lq, next, &len);
    msum += lq->mf;
    free(lq);
  }
  *mf = msum;
  return len;
}

/* shrink a partition's word range past all-visited words at both ends */
static void shrink(const hb_ws* ws, int64_t* lo, int64_t* hi) {
  while (*lo < *hi && ws->visited[*lo] == ~0ull) ++*lo;
  while (*hi > *lo && ws->visited[*hi - 1] == ~0ull) --*hi;
}

/* Algorithm 6: bitmap cur -> bitmap next; returns |F_next|, *mf its degree
 * sum, *exam the edges examined. */
static int64_t bottom_up(hb_ws* ws, const uint64_t* cur, uint64_t* next, int32_t L1,
                         int64_t* mf, int64_t* exam) {
  int64_t s = 0, nn = 0, msum = 0, ex = 0;
  const int t = ws->t;
  memset(next, 0, (size_t)ws->words * 8);
#pragma omp parallel num_threads(t) reduction(+ : nn, msum, ex)
  {
    for (;;) {
      const int64_t pos = __atomic_fetch_add(&s, 1, __ATOMIC_RELAXED);
      if (pos >= ws->nparts) break;
      int64_t lo = ws->part_lo[pos], hi = ws->part_hi[pos];
      shrink(ws, &lo, &hi);
      /* neighbors+: the highest-degree neighbour, the row's last entry */
      for (int64_t w = lo; w < hi; ++w) {
        uint64_t unv = ~ws->visited[w], found = 0;
        while (unv) {
          const int bit = __builtin_ctzll(unv);
          unv &= unv - 1;
          const int64_t v = w * 64 + bit;
          if (v >= ws->nb) break;
          const int64_t b = ws->off[v], e = ws->off[v + 1];
          if (e == b) continue;
          ex += 1;
          const int32_t x = ws->col[e - 1];
          if (bit_of(cur, x)) {
            ws->pi[v] = x;
            ws->lev[v] = L1;
            found |= 1ull << bit;
            nn += 1;
            msum += e - b;
          }
        }
        next[w] = found;
      }
      or_128(ws->visited, next, lo, hi);
      shrink(ws, &lo, &hi);
      /* neighbors-: the rest in decreasing degree (the row read backwards) */
      for (int64_t w = lo; w < hi; ++w) {
        uint64_t unv = ~ws->visited[w], found = 0;
        while (unv) {
          const int bit = __builtin_ctzll(unv);
          unv &= unv - 1;
          const int64_t v = w * 64 + bit;
          if (v >= ws->nb) break;
          const int64_t b = ws->off[v], e = ws->off[v + 1];
          for (int64_t k = e - 2; k >= b; --k) {
            ex += 1;
            const int32_t x = ws->col[k];
            if (bit_of(cur, x)) {
              ws->pi[v] = x;
              ws->lev[v] = L1;
              found |= 1ull << bit;
              nn += 1;
              msum += e - b;
              break;
            }
          }
        }
        next[w] |= found;
      }
      or_128(ws->visited, next, lo, hi);
      ws->part_lo[pos] = lo;
      ws->part_hi[pos] = hi;
    }
  }
  *mf = msum;
  *exam = ex;
  return nn;
}

/* queue -> bitmap (before a bottom-up step that follows a top-down one) */
static void q_to_bm(hb_ws* ws, const int32_t* q, int64_t nf, uint64_t* bm) {
  memset(bm, 0, (size_t)ws->words * 8);
#pragma omp parallel for num_threads(ws->t) schedule(static)
  for (int64_t j = 0; j < nf; ++j)
    __atomic_fetch_or(&bm[q[j] >> 6], 1ull << (q[j] & 63), __ATOMIC_RELAXED);
}

/* bitmap -> queue (before a top-down step that follows a bottom-up one) */
static int64_t bm_to_q(hb_ws* ws, const uint64_t* bm, int32_t* q) {
  int64_t len = 0;
#pragma omp parallel num_threads(ws->t)
  {
    local_q* lq = (local_q*)malloc(sizeof(local_q));
    lq->cnt = 0;
#pragma omp for schedule(static)
    for (int64_t w = 0; w < ws->words; ++w) {
      uint64_t x = bm[w];
      while (x) {
        const int bit = __builtin_ctzll(x);
        x &= x - 1;
        lq->buf[lq->cnt++] = (int32_t)(w * 64 + bit);
        if (lq->cnt == HB_LOCAL) lq_flush(lq, q, &len);
      }
    }
    lq_flush(lq, q, &len);
    free(lq);
  }
  return len;
}

/* ------------------------------------------------------------ search */

/* BFS from `root` (original ID). parent, level: n entries, original IDs,
 * -1 where unreached (an isolated root reaches only itself). Returns 0, or
 * -1 for a bad root / options. */
int32_t hb_bfs(hb_ws* ws, int32_t root, const hb_opts* o, int32_t* parent, int32_t* level,
               hb_stats* st) {
  if (!ws || root < 0 || root >= ws->n || !parent || !level) return -1;
  const int32_t alpha = o && o->alpha > 0 ? o->alpha : 14;
  const int32_t beta = o && o->beta > 0 ? o->beta : 24;
  const int td_kind = o ? o->td_kind : 0;
  const int32_t nb = ws->nb;
  const int64_t nnz = nb > 0 ? ws->off[nb] : 0;
  hb_stats S;
  memset(&S, 0, sizeof(S));
  S.threads = ws->t;
  memset(ws->visited, 0, (size_t)ws->words * 8);
  /* bits past nb count as visited, so shrinking and bottom-up skip them */
  for (int64_t v = nb; v < ws->words * 64; ++v) ws->visited[v >> 6] |= 1ull << (v & 63);
  for (int64_t k = 0; k < ws->nparts; ++k) {
    ws->part_lo[k] = ws->part_base[k] * HB_BLOCK_WORDS;
    ws->part_hi[k] = ws->part_base[k + 1] * HB_BLOCK_WORDS;
  }
  const int32_t r = ws->new_of_old ? ws->new_of_old[root] : root;
  int64_t nf = 0, mf = 0, nvis = 0, mvis = 0;
  int queue = 1, dir = 0, seen_bu = 0;
  int32_t *qc = ws->qa, *qn = ws->qb;
  uint64_t *bc = ws->fa, *bn = ws->fb;
  if (r >= 0 && r < nb) {
    ws->visited[r >> 6] |= 1ull << (r & 63);
    ws->pi[r] = r;
    ws->lev[r] = 0;
    qc[0] = r;
    nf = 1;
    mf = ws->off[r + 1] - ws->off[r];
    nvis = 1;
    mvis = mf;
  }
  int32_t L = 0;
  while (nf > 0) {
    int64_t nn, mn;
    if (dir == 0) {
      if (!queue) {
        nf = bm_to_q(ws, bc, qc);
        queue = 1;
      }
      const int alg4 = td_kind == 1 || (td_kind == 0 && !seen_bu);
      nn = top_down(ws, qc, nf, qn, L + 1, alg4, &mn);
      int32_t* tq = qc;
      qc = qn;
      qn = tq;
      S.td_levels++;
    } else {
      if (queue) {
        q_to_bm(ws, qc, nf, bc);
        queue = 0;
      }
      int64_t ex = 0;
      nn = bottom_up(ws, bc, bn, L + 1, &mn, &ex);
      S.bu_examined += ex;
      uint64_t* tb = bc;
      bc = bn;
      bn = tb;
      seen_bu = 1;
      S.bu_levels++;
    }
    const int64_t prev_nf = nf;
    nf = nn;
    mf = mn;
    nvis += nf;
    mvis += mf;
    const int64_t nu = nb - nvis, mu = nnz - mvis;
    (void)nu;
    if (dir == 0) {
      dir = (mf * (int64_t)alpha > mu) ? 1 : 0;
    } else {
      dir = (nf < prev_nf && nf * (int64_t)beta < (int64_t)nb) ? 0 : 1;
    }
    ++L;
  }
  S.levels = L;
  /* outputs in original IDs */
  const int32_t n = ws->n;
#pragma omp parallel for num_threads(ws->t) schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    const int32_t x = ws->new_of_old ? ws->new_of_old[v] : (int32_t)v;
    if (x >= 0 && x < nb && bit_of(ws->visited, x)) {
      const int32_t p = ws->pi[x];
      parent[v] = ws->old_of_new ? ws->old_of_new[p] : p;
      level[v] = ws->lev[x];
    } else {
      parent[v] = -1;
      level[v] = -1;
    }
  }
  parent[root] = root;
  level[root] = 0;
  if (st) *st = S;
  return 0;
}
