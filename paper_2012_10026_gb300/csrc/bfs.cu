// Hybrid breadth-first search (Algorithm 2) on the graph's current CSR.
//
// Per level L the frontier F_L is either a queue (after a top-down level) or
// a bitmap (after a bottom-up level). A one-warp controller kernel decides
// the direction of every level on the device from the frontier statistics;
// the host reads the decision back (one small copy per level) and launches:
//
//   top-down (Algorithms 1 and 4): td_front walks the queue one thread per
//     vertex; vertices with degree < t1 are expanded on the spot, the others
//     go to three bins expanded by one warp (t1 <= deg < t2), one CTA
//     (t2 <= deg < t3) or the whole grid (deg >= t3) -- the GPU form of
//     Algorithm 4's even split of a long neighbour list over all threads.
//     Neighbour lists are read with aligned 128-bit loads. A neighbour is
//     claimed by an atomicOr on its word of the visited bitmap; the winner
//     writes (parent, level) and appends it to the next queue through a
//     per-warp shared-memory buffer (one global atomic per ~224 vertices).
//   bottom-up (Algorithms 5 and 6): one warp per pair of 32-vertex words of
//     the visited bitmap; each unvisited vertex scans its row until the first
//     neighbour whose bit is set in the current-frontier bitmap (early break).
//     The first probe of both words is issued before any continuation so that
//     each lane keeps two independent load chains in flight. Rows are scanned
//     from their end by default: under RCM labels grow with degree, so this is
//     Algorithm 6's highest-degree-first order. The word's owner writes the
//     next-frontier word and ORs it into visited (no atomics: the paper's
//     "visited |= F_next" folded into the same pass).
//
// Statistics of the next frontier (size, degree sum, label range, degree
// histogram, edges examined) are reduced per block and added with one atomic
// per block. (parent, level) of BFS-graph vertices are kept packed as int2 and
// are only meaningful where the visited bit is set, so nothing but the
// visited bitmap is cleared per search.
#include <math.h>
#include <string.h>

#include "g3_prims.cuh"

// Device-side controller record; mirrored to pinned host memory each level.
struct Ctrl {
  // accumulators for the frontier being produced (reset by the controller)
  unsigned long long q_len;     // top-down: next queue length
  unsigned long long nx_nf;     // bottom-up: next frontier size
  unsigned long long nx_mf;     // sum of degrees of the next frontier
  unsigned long long nx_exam;   // bottom-up: edges examined
  unsigned long long nx_hist[4];
  unsigned int nx_min, nx_max;
  unsigned long long bin_len[4];  // top-down bins of the current level
  unsigned long long g_pack;      // grid bin: slots << 38 | edge total
  unsigned long long conv_len;    // bitmap -> queue conversion length
  // current frontier F_L and its decision
  long long nf, mf, nu, mu, exam_prev;
  long long hist[4];
  int id_min, id_max;
  int level;
  int dir;
  int t1, t2, t3;
  float mlp_out[4];
  long long prev_nf;
  long long n_visited, m_visited;
};

struct g3_bfs_ws {
  int32_t nb;
  int64_t nwords;
  uint32_t *visited, *fa, *fb, *vis_save;
  int32_t *qa, *qb, *bins;  // bins: 3 segments of nb entries (warp, CTA, grid)
  int64_t* goff;            // edge offset of each grid-bin vertex
  int2* pl;                 // (parent, level) per BFS-graph vertex
  int32_t *out_parent, *out_level;  // staging for host outputs (n entries)
  unsigned* bcount;                 // translation: entries per window
  unsigned long long* bucket;       // translation: TR_W slots per window
  int64_t nbuckets;
  Ctrl* ctrl;
  Ctrl* h_ctrl;  // pinned
  cudaEvent_t ev[6];
  // resident-grid sizes (SMs x blocks per SM) per kernel
  int grid_front, grid_bins, grid_bu, grid_conv, grid_tr, grid_trb, grid_trw;
};

void g3_bfs_ws_free(g3_bfs_ws* ws) {
  if (!ws) return;
  void* all[] = {ws->visited, ws->fa,  ws->fb,         ws->vis_save,  ws->qa,  ws->qb,
                 ws->bins,    ws->pl,  ws->out_parent, ws->out_level, ws->ctrl, ws->goff,
                 ws->bcount,  ws->bucket};
  for (void* p : all)
    if (p) cudaFree(p);
  if (ws->h_ctrl) cudaFreeHost(ws->h_ctrl);
  for (int i = 0; i < 6; ++i)
    if (ws->ev[i]) cudaEventDestroy(ws->ev[i]);
  free(ws);
}

// ----------------------------------------------------------- device helpers
__device__ __forceinline__ int deg_bucket(int64_t d) {
  return d < 32 ? 0 : (d < 1024 ? 1 : (d < 32768 ? 2 : 3));
}

// Per-thread statistics in 32-bit registers (a thread sees far fewer than
// 2^32 vertices or edges per launch); reduced per block in 64 bits.
struct StatAcc {
  unsigned nf, mf, ex, h0, h1, h2, h3, mn, mx;
  __device__ void init() {
    nf = mf = ex = h0 = h1 = h2 = h3 = 0;
    mn = 0xFFFFFFFFu;
    mx = 0;
  }
  __device__ void add_vertex(int32_t v, int64_t d) {
    nf++;
    mf += (unsigned)d;
    int b = deg_bucket(d);
    h0 += b == 0;
    h1 += b == 1;
    h2 += b == 2;
    h3 += b == 3;
    mn = min(mn, (unsigned)v);
    mx = max(mx, (unsigned)v);
  }
  __device__ void flush(Ctrl* c) {
    __shared__ unsigned long long s[8][7];
    __shared__ unsigned int smn[8], smx[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long v[7] = {nf, mf, ex, h0, h1, h2, h3};
    unsigned a = mn, b = mx;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane == 0) {
      for (int k = 0; k < 7; ++k) s[warp][k] = v[k];
      smn[warp] = a;
      smx[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t[7] = {0, 0, 0, 0, 0, 0, 0};
      unsigned tmn = 0xFFFFFFFFu, tmx = 0;
      for (int w = 0; w < nw; ++w) {
        for (int k = 0; k < 7; ++k) t[k] += s[w][k];
        tmn = min(tmn, smn[w]);
        tmx = max(tmx, smx[w]);
      }
      if (t[0]) atomicAdd(&c->nx_nf, t[0]);
      if (t[1]) atomicAdd(&c->nx_mf, t[1]);
      if (t[2]) atomicAdd(&c->nx_exam, t[2]);
      for (int k = 0; k < 4; ++k)
        if (t[3 + k]) atomicAdd(&c->nx_hist[k], t[3 + k]);
      if (t[0]) {
        atomicMin(&c->nx_min, tmn);
        atomicMax(&c->nx_max, tmx);
      }
    }
  }
};

__device__ __forceinline__ bool td_claim(uint32_t* visited, int32_t w) {
  const uint32_t bit = 1u << (w & 31);
  uint32_t* word = &visited[w >> 5];
  if (__ldcg(word) & bit) return false;
  return !(atomicOr(word, bit) & bit);
}

__device__ __forceinline__ void reset_next(Ctrl* c) {
  c->q_len = 0;
  c->nx_nf = 0;
  c->nx_mf = 0;
  c->nx_exam = 0;
  for (int k = 0; k < 4; ++k) {
    c->nx_hist[k] = 0;
    c->bin_len[k] = 0;
  }
  c->nx_min = 0xFFFFFFFFu;
  c->nx_max = 0;
  c->g_pack = 0;
  c->conv_len = 0;
}

// ------------------------------------------------------------------- init
// Sets up F_0 = {root} (root_new < 0 or >= nb: no BFS-graph vertex). The
// visited bitmap has been cleared on the stream before.
__global__ void bfs_root(const int32_t* new_of_old, int32_t root, int32_t nb, int64_t nnz,
                         const int64_t* off, uint32_t* visited, int2* pl, int32_t* q, Ctrl* c,
                         int t1, int t2, int t3) {
  int32_t r = new_of_old ? new_of_old[root] : root;
  memset(c, 0, sizeof(Ctrl));
  reset_next(c);
  c->t1 = t1;
  c->t2 = t2;
  c->t3 = t3;
  c->dir = G3_DIR_TD;  // Algorithm 2 starts top-down
  if (r < 0 || r >= nb) {
    c->nf = 0;
    c->nu = nb;
    c->mu = nnz;
    return;
  }
  visited[r >> 5] |= 1u << (r & 31);
  pl[r] = make_int2(r, 0);
  q[0] = r;
  long long d = off[r + 1] - off[r];
  c->nf = 1;
  c->mf = d;
  c->hist[deg_bucket(d)] = 1;
  c->id_min = c->id_max = r;
  c->n_visited = 1;
  c->m_visited = d;
  c->nu = nb - 1;
  c->mu = nnz - d;
  c->prev_nf = 0;
}

// --------------------------------------------------------------- top-down
struct TdArgs {
  const int64_t* off;
  const int32_t* col;
  uint32_t* visited;
  int2* pl;
  int32_t lnext;
  int32_t* qnext;
  Ctrl* c;
};

// Per-warp staging of the next queue in shared memory: claimed vertices are
// compacted into the warp's buffer with a ballot and written to the global
// queue in one coalesced burst, reserving space with one atomic per ~224
// vertices instead of one per warp step (the queue counter is a single
// address that every warp of the grid would otherwise hit).
#define WQ_CAP 256
#define WQ_FLUSH (WQ_CAP - 32)
struct WarpQueue {
  int32_t* buf;  // this warp's WQ_CAP-entry shared buffer
  int cnt;       // warp-uniform fill level
};

__device__ __forceinline__ void wq_flush(WarpQueue& q, int32_t* gq, unsigned long long* glen) {
  if (q.cnt == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(glen, (unsigned long long)q.cnt);
  base = __shfl_sync(0xffffffffu, base, 0);
  __syncwarp();
  for (int i = lane; i < q.cnt; i += 32) gq[base + i] = q.buf[i];
  __syncwarp();
  q.cnt = 0;
}

// All 32 lanes call it together.
__device__ __forceinline__ void wq_push(WarpQueue& q, bool want, int32_t item, int32_t* gq,
                                        unsigned long long* glen) {
  const unsigned bal = __ballot_sync(0xffffffffu, want);
  if (bal == 0) return;
  if (want) q.buf[q.cnt + __popc(bal & g3_lanemask_lt())] = item;
  q.cnt += __popc(bal);
  __syncwarp();
  if (q.cnt > WQ_FLUSH) wq_flush(q, gq, glen);
}

#define WQ_DECLARE(q)                                      \
  __shared__ int32_t wq_mem[8][WQ_CAP];                    \
  WarpQueue q{wq_mem[threadIdx.x >> 5], 0}

// Claims w for v and records the statistics of the claimed vertex (the next
// frontier's degree sum, label range and histogram). All 32 lanes must call
// it together.
__device__ __forceinline__ void td_visit(const TdArgs& a, WarpQueue& q, StatAcc& acc, bool has,
                                         int32_t w, int32_t v) {
  bool claim = has && td_claim(a.visited, w);
  if (claim) {
    a.pl[w] = make_int2(v, a.lnext);
    acc.add_vertex(w, a.off[w + 1] - a.off[w]);
  }
  wq_push(q, claim, w, a.qnext, &a.c->q_len);
}

// Processes row entries [b, e) of vertex v with `nthr` cooperating threads
// (index t), four entries per thread per step through aligned 128-bit loads.
// Every lane of each participating warp runs the same number of steps.
__device__ __forceinline__ void td_row_vec4(const TdArgs& a, WarpQueue& q, StatAcc& acc,
                                            int32_t v, int64_t b, int64_t e, int64_t t,
                                            int64_t nthr, int64_t steps) {
  const int64_t a0 = b & ~3ll;
  for (int64_t s = 0; s < steps; ++s) {
    const int64_t j = a0 + 4 * (t + s * nthr);
    int4 x = make_int4(0, 0, 0, 0);
    if (j < e) x = *reinterpret_cast<const int4*>(a.col + j);
    td_visit(a, q, acc, j + 0 >= b && j + 0 < e, x.x, v);
    td_visit(a, q, acc, j + 1 >= b && j + 1 < e, x.y, v);
    td_visit(a, q, acc, j + 2 >= b && j + 2 < e, x.z, v);
    td_visit(a, q, acc, j + 3 >= b && j + 3 < e, x.w, v);
  }
}

// Grid-bin slots and their edge offsets are handed out by one 64-bit atomic
// (slot count in the high bits, edge total in the low 38 bits), so the offsets
// ascend with the slot index.
#define GP_SHIFT 38
#define GP_MASK ((1ull << GP_SHIFT) - 1ull)

// Thread per frontier vertex: degree < t1 expanded here, larger degrees
// binned (warp / CTA / grid).
__global__ void __launch_bounds__(256) td_front(TdArgs a, const int32_t* __restrict__ q,
                                                int64_t qlen, int32_t* bins, int64_t* goff,
                                                int64_t nb1) {
  const int t1 = a.c->t1, t2 = a.c->t2, t3 = a.c->t3;
  WQ_DECLARE(wq);
  StatAcc acc;
  acc.init();
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < qlen;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool act = i < qlen;
    int32_t v = act ? q[i] : 0;
    int64_t b = act ? a.off[v] : 0, e = act ? a.off[v + 1] : 0, d = e - b;
    bool small = act && d < t1;
    int bin = !act || small ? -1 : (d < t2 ? 0 : (d < t3 ? 1 : 2));
    for (int k = 0; k < 2; ++k)
      g3_warp_append(0xffffffffu, bin == k, v, bins + k * nb1, &a.c->bin_len[1 + k]);
    if (bin == 2) {
      const unsigned long long old =
          atomicAdd(&a.c->g_pack, (1ull << GP_SHIFT) | (unsigned long long)d);
      const int64_t slot = (int64_t)(old >> GP_SHIFT);
      bins[2 * nb1 + slot] = v;
      goff[slot] = (int64_t)(old & GP_MASK);
    }
    const int cnt = small ? (int)d : 0;
    const int maxc = __reduce_max_sync(0xffffffffu, cnt);
    for (int k = 0; k < maxc; ++k) {
      bool has = k < cnt;
      int32_t w = has ? a.col[b + k] : 0;
      td_visit(a, wq, acc, has, w, v);
    }
  }
  wq_flush(wq, a.qnext, &a.c->q_len);
  acc.flush(a.c);
}

// The three bins in one launch: warp per warp-bin vertex, CTA per CTA-bin
// vertex, and the grid bin as one flattened edge range split evenly over all
// warps of the grid (Algorithm 4's even split, applied to every hub at once).
__global__ void __launch_bounds__(256) td_bins(TdArgs a, const int32_t* __restrict__ bins,
                                               const int64_t* __restrict__ goff, int64_t nb1) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  WQ_DECLARE(wq);
  StatAcc acc;
  acc.init();
  const int64_t len1 = (int64_t)a.c->bin_len[1];
  for (int64_t i = gw; i < len1; i += nwarps) {
    int32_t v = bins[i];
    int64_t b = a.off[v], e = a.off[v + 1];
    int64_t steps = (e - (b & ~3ll) + 127) / 128;
    td_row_vec4(a, wq, acc, v, b, e, lane, 32, steps);
  }
  const int64_t len2 = (int64_t)a.c->bin_len[2];
  for (int64_t i = blockIdx.x; i < len2; i += gridDim.x) {
    int32_t v = bins[nb1 + i];
    int64_t b = a.off[v], e = a.off[v + 1];
    int64_t steps = (e - (b & ~3ll) + 4 * blockDim.x - 1) / (4 * blockDim.x);
    td_row_vec4(a, wq, acc, v, b, e, threadIdx.x, blockDim.x, steps);
  }
  const unsigned long long gp = a.c->g_pack;
  const int64_t nh = (int64_t)(gp >> GP_SHIFT), E = (int64_t)(gp & GP_MASK);
  if (E > 0) {
    const int32_t* gbin = bins + 2 * nb1;
    const int64_t per = (((E + nwarps - 1) / nwarps) + 31) & ~31ll;
    const int64_t j0 = gw * per, j1 = min(E, j0 + per);
    if (j0 < j1) {
      int64_t h = g3_upper_bound_i64(goff, nh, j0) - 1;
      for (int64_t base = j0; base < j1; base += 32) {
        const int64_t j = base + lane;
        const bool act = j < j1;
        int32_t v = 0, w = 0;
        if (act) {
          while (h + 1 < nh && goff[h + 1] <= j) ++h;
          v = gbin[h];
          w = a.col[a.off[v] + (j - goff[h])];
        }
        td_visit(a, wq, acc, act, w, v);
      }
    }
  }
  wq_flush(wq, a.qnext, &a.c->q_len);
  acc.flush(a.c);
}

// -------------------------------------------------------------- bottom-up
__device__ __forceinline__ bool in_frontier(const uint32_t* __restrict__ f, int32_t w) {
  return (__ldg(&f[w >> 5]) >> (w & 31)) & 1u;
}

// Scans the rest of a row after a missed first probe; returns the parent or
// -1 and advances k (edges examined).
template <int REV>
__device__ __forceinline__ int32_t bu_scan_rest(const int32_t* __restrict__ col,
                                                const uint32_t* __restrict__ fcur, int64_t b,
                                                int64_t e, int64_t& k) {
  const int64_t d = e - b;
  while (k < d) {
    const int32_t w = col[REV ? e - 1 - k : b + k];
    ++k;
    if (in_frontier(fcur, w)) return w;
  }
  return -1;
}

template <int REV>
__global__ void __launch_bounds__(256) bu_pull(int32_t nb, int64_t nwords, uint32_t* visited,
                                               const uint32_t* __restrict__ fcur,
                                               uint32_t* __restrict__ fnext,
                                               const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ col, int2* pl,
                                               int32_t lnext, Ctrl* c) {
  StatAcc acc;
  acc.init();
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t w0 = 2 * wid; w0 < nwords; w0 += 2 * nwarps) {
    const bool has1 = w0 + 1 < nwords;
    const uint32_t vis0 = visited[w0];
    const uint32_t vis1 = has1 ? visited[w0 + 1] : 0xFFFFFFFFu;
    const int64_t v0 = w0 * 32 + lane, v1 = v0 + 32;
    const bool c0 = v0 < nb && !((vis0 >> lane) & 1u);
    const bool c1 = v1 < nb && !((vis1 >> lane) & 1u);
    if (!__any_sync(0xffffffffu, c0 || c1)) {
      if (lane == 0) {
        fnext[w0] = 0u;
        if (has1) fnext[w0 + 1] = 0u;
      }
      continue;
    }
    int64_t b0 = 0, e0 = 0, b1 = 0, e1 = 0;
    if (c0) {
      b0 = off[v0];
      e0 = off[v0 + 1];
    }
    if (c1) {
      b1 = off[v1];
      e1 = off[v1 + 1];
    }
    // first probes of both vertices, independent of each other
    int32_t x0 = -1, x1 = -1;
    if (e0 > b0) x0 = col[REV ? e0 - 1 : b0];
    if (e1 > b1) x1 = col[REV ? e1 - 1 : b1];
    int32_t p0 = (x0 >= 0 && in_frontier(fcur, x0)) ? x0 : -1;
    int32_t p1 = (x1 >= 0 && in_frontier(fcur, x1)) ? x1 : -1;
    int64_t k0 = e0 > b0 ? 1 : 0, k1 = e1 > b1 ? 1 : 0;
    if (p0 < 0) p0 = bu_scan_rest<REV>(col, fcur, b0, e0, k0);
    if (p1 < 0) p1 = bu_scan_rest<REV>(col, fcur, b1, e1, k1);
    acc.ex += (unsigned)(k0 + k1);
    const uint32_t n0 = __ballot_sync(0xffffffffu, p0 >= 0);
    const uint32_t n1 = __ballot_sync(0xffffffffu, p1 >= 0);
    if (p0 >= 0) {
      pl[v0] = make_int2(p0, lnext);
      acc.add_vertex((int32_t)v0, e0 - b0);
    }
    if (p1 >= 0) {
      pl[v1] = make_int2(p1, lnext);
      acc.add_vertex((int32_t)v1, e1 - b1);
    }
    if (lane == 0) {
      fnext[w0] = n0;
      if (n0) visited[w0] = vis0 | n0;
      if (has1) {
        fnext[w0 + 1] = n1;
        if (n1) visited[w0 + 1] = vis1 | n1;
      }
    }
  }
  acc.flush(c);
}

// ------------------------------------------------------------ conversions
__global__ void q_to_bitmap(const int32_t* __restrict__ q, int64_t len, uint32_t* bm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = q[i];
    atomicOr(&bm[v >> 5], 1u << (v & 31));
  }
}

__global__ void bitmap_to_q(const uint32_t* __restrict__ bm, int64_t nwords, int32_t* q,
                            unsigned long long* len) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
       base < nwords; base += nwarps * 32) {
    const int64_t w = base + lane;
    uint32_t bits = w < nwords ? bm[w] : 0u;
    unsigned c = __popc(bits), inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const unsigned total = __shfl_sync(0xffffffffu, inc, 31);
    if (total == 0) continue;
    unsigned long long start = 0;
    if (lane == 31) start = atomicAdd(len, (unsigned long long)total);
    start = __shfl_sync(0xffffffffu, start, 31);
    unsigned long long p = start + inc - c;
    while (bits) {
      int b = __ffs(bits) - 1;
      q[p++] = (int32_t)(w * 32 + b);
      bits &= bits - 1u;
    }
  }
}

// ------------------------------------------------------------- controller
// Learned controller: 12-32-4 MLP (ReLU) evaluated by one warp, lane j =
// hidden unit j. Parameter layout: W1[32][12], b1[32], W2[4][32], b2[4].
__device__ void mlp_features(const Ctrl* c, int32_t nb, int prev_dir, float* f) {
  const float nf = (float)c->nf, mf = (float)c->mf, nu = (float)c->nu, mu = (float)c->mu;
  f[0] = log2f(1.f + nf);
  f[1] = log2f(1.f + mf);
  f[2] = log2f(1.f + nu);
  f[3] = log2f(1.f + mu);
  f[4] = (c->nf > 0 && nb > 0) ? (float)(c->id_max - c->id_min) / (float)nb : 0.f;
  f[5] = log2f((1.f + mf) / (1.f + mu));
  f[6] = (float)c->level / 32.f;
  f[7] = (float)prev_dir;
  const float tot = c->nf > 0 ? (float)c->nf : 1.f;
  for (int k = 0; k < 4; ++k) f[8 + k] = (float)c->hist[k] / tot;
}

__device__ void mlp_eval_warp(const float* __restrict__ P, const float* f, float* out) {
  const int j = threadIdx.x & 31;
  const float* W1 = P;
  const float* b1 = P + 32 * 12;
  const float* W2 = b1 + 32;
  const float* b2 = W2 + 4 * 32;
  float z = b1[j];
#pragma unroll
  for (int i = 0; i < 12; ++i) z = fmaf(W1[j * 12 + i], f[i], z);
  const float h = fmaxf(z, 0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float s = W2[k * 32 + j] * h;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    out[k] = s + b2[k];
  }
}

__device__ __forceinline__ int clamp_thr(float lg, int lo, int hi) {
  float x = fminf(fmaxf(rintf(lg), (float)lo), (float)hi);
  return 1 << (int)x;
}

// After the expansion of level L: promote the produced frontier to F_{L+1},
// update the visited totals, decide its direction and clear the accumulators
// for the next expansion.
__global__ void bfs_control(Ctrl* c, int32_t nb, int64_t nnz, int controller, int alpha,
                            int beta, const float* __restrict__ mlp, int t1d, int t2d, int t3d,
                            int was_td) {
  __shared__ float feat[12];
  __shared__ int decide;
  const int lane = threadIdx.x;
  if (lane == 0) {
    const int prev_dir = c->dir;
    const long long prev_nf = c->nf;
    const long long nf = was_td ? (long long)c->q_len : (long long)c->nx_nf;
    c->exam_prev = (long long)c->nx_exam;
    c->nf = nf;
    c->mf = (long long)c->nx_mf;
    for (int k = 0; k < 4; ++k) c->hist[k] = (long long)c->nx_hist[k];
    c->id_min = nf ? (int)c->nx_min : 0;
    c->id_max = nf ? (int)c->nx_max : 0;
    c->n_visited += nf;
    c->m_visited += c->mf;
    c->nu = nb - c->n_visited;
    c->mu = nnz - c->m_visited;
    c->level += 1;
    c->prev_nf = prev_nf;
    int d;
    if (controller == G3_CTRL_TOPDOWN) {
      d = G3_DIR_TD;
    } else if (controller == G3_CTRL_BOTTOMUP) {
      d = G3_DIR_BU;
    } else if (prev_dir == G3_DIR_TD) {
      d = (c->mf * (long long)alpha > c->mu) ? G3_DIR_BU : G3_DIR_TD;
    } else {
      d = (nf < prev_nf && nf * (long long)beta < (long long)nb) ? G3_DIR_TD : G3_DIR_BU;
    }
    c->t1 = t1d;
    c->t2 = t2d;
    c->t3 = t3d;
    decide = d;
    if (controller == G3_CTRL_LEARNED) mlp_features(c, nb, prev_dir, feat);
    reset_next(c);
  }
  __syncwarp();
  if (controller == G3_CTRL_LEARNED) {
    float out[4];
    mlp_eval_warp(mlp, feat, out);
    if (lane == 0) {
      for (int k = 0; k < 4; ++k) c->mlp_out[k] = out[k];
      decide = out[0] < 0.f ? G3_DIR_BU : G3_DIR_TD;
      int a1 = clamp_thr(out[1], 2, 12), a2 = clamp_thr(out[2], 6, 18),
          a3 = clamp_thr(out[3], 10, 26);
      if (a2 <= a1) a2 = a1 * 2;
      if (a3 <= a2) a3 = a2 * 2;
      c->t1 = a1;
      c->t2 = a2;
      c->t3 = a3;
    }
    __syncwarp();
  }
  if (lane == 0) c->dir = decide;
}

// --------------------------------------------------------- output mapping
__global__ void bfs_translate(int32_t n, int32_t nb, int32_t root,
                              const int32_t* __restrict__ new_of_old,
                              const int32_t* __restrict__ old_of_new,
                              const uint32_t* __restrict__ visited,
                              const int2* __restrict__ pl, int32_t* parent, int32_t* level) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = -1, l = -1;
    const int32_t x = new_of_old ? new_of_old[v] : (int32_t)v;
    if (x < nb && ((__ldg(&visited[x >> 5]) >> (x & 31)) & 1u)) {
      const int2 t = pl[x];
      p = old_of_new ? old_of_new[t.x] : t.x;
      l = t.y;
    }
    if (v == root) {
      p = root;
      l = 0;
    }
    parent[v] = p;
    level[v] = l;
  }
}

// Output translation of a relabelled graph in two streaming passes instead of
// one random gather per vertex. The original IDs are cut into windows of
// TR_W; pass 1 walks the BFS-graph labels in order (coalesced) and appends
// each reached vertex to its window's bucket (one counter atomic, writes
// that stay sequential per bucket); pass 2 gives each window to one block,
// which assembles the window's parent[] and level[] in shared memory (-1 for
// unreached) and writes them out coalesced.
#define TR_SHIFT 12
#define TR_W (1 << TR_SHIFT)
#define TR_LEVEL_BITS 20

__global__ void tr_bucket(int32_t nb, const uint32_t* __restrict__ visited,
                          const int2* __restrict__ pl, const int32_t* __restrict__ old_of_new,
                          unsigned* bcount, unsigned long long* bucket) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nb;
       x += (int64_t)gridDim.x * blockDim.x) {
    if (!((__ldg(&visited[x >> 5]) >> (x & 31)) & 1u)) continue;
    const int2 t = pl[x];
    const int32_t o = old_of_new[x];
    const int32_t po = __ldg(&old_of_new[t.x]);
    const int64_t b = o >> TR_SHIFT;
    const unsigned slot = atomicAdd(&bcount[b], 1u);
    bucket[b * TR_W + slot] = ((unsigned long long)(o & (TR_W - 1)) << 52) |
                              ((unsigned long long)(t.y & ((1 << TR_LEVEL_BITS) - 1)) << 32) |
                              (unsigned)po;
  }
}

__global__ void __launch_bounds__(256) tr_window(int32_t n, int32_t root,
                                                 const unsigned* __restrict__ bcount,
                                                 const unsigned long long* __restrict__ bucket,
                                                 int32_t* parent, int32_t* level) {
  __shared__ int32_t sp[TR_W], sl[TR_W];
  const int64_t nbk = ((int64_t)n + TR_W - 1) >> TR_SHIFT;
  for (int64_t b = blockIdx.x; b < nbk; b += gridDim.x) {
    const int64_t base = b << TR_SHIFT;
    for (int i = threadIdx.x; i < TR_W; i += blockDim.x) {
      sp[i] = -1;
      sl[i] = -1;
    }
    __syncthreads();
    const unsigned cnt = bcount[b];
    for (unsigned i = threadIdx.x; i < cnt; i += blockDim.x) {
      const unsigned long long e = bucket[base + i];
      const int lo = (int)(e >> 52);
      sp[lo] = (int32_t)(unsigned)(e & 0xFFFFFFFFull);
      sl[lo] = (int32_t)((e >> 32) & ((1u << TR_LEVEL_BITS) - 1));
    }
    __syncthreads();
    if (threadIdx.x == 0 && root >= base && root < base + TR_W) {
      sp[root - base] = root;  // also an isolated root
      sl[root - base] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TR_W && base + i < n; i += blockDim.x) {
      parent[base + i] = sp[i];
      level[base + i] = sl[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host
extern "C" void g3_bfs_opts_default(g3_bfs_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->controller = G3_CTRL_HEURISTIC;
  o->alpha = 14;
  o->beta = 24;
  o->t1 = 32;
  o->t2 = 1024;
  o->t3 = 32768;
  o->bu_reverse = 1;
}

template <class K>
static int resident_grid(K kernel, int block) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0);
  cudaGetLastError();
  if (sms < 1) sms = G3_NUM_SMS;
  if (per < 1) per = 1;
  return sms * per;
}

static g3_status ws_create(g3_graph* g, g3_bfs_ws** out) {
  g3_bfs_ws* ws = (g3_bfs_ws*)calloc(1, sizeof(g3_bfs_ws));
  if (!ws) return G3_ENOMEM;
  ws->nb = g->n_bfs;
  ws->nwords = ((int64_t)g->n_bfs + 31) / 32;
  const size_t nb1 = (size_t)g->n_bfs + 4, nw = (size_t)ws->nwords + 4, n1 = (size_t)g->n + 4;
  struct {
    void** p;
    size_t bytes;
  } req[] = {
      {(void**)&ws->visited, nw * 4},     {(void**)&ws->fa, nw * 4},
      {(void**)&ws->fb, nw * 4},          {(void**)&ws->vis_save, nw * 4},
      {(void**)&ws->qa, nb1 * 4},         {(void**)&ws->qb, nb1 * 4},
      {(void**)&ws->bins, nb1 * 4 * 3},   {(void**)&ws->pl, nb1 * 8},
      {(void**)&ws->goff, nb1 * 8},
      {(void**)&ws->out_parent, n1 * 4},  {(void**)&ws->out_level, n1 * 4},
      {(void**)&ws->bcount, ((size_t)(g->n >> TR_SHIFT) + 2) * 4},
      {(void**)&ws->bucket, ((size_t)(g->n >> TR_SHIFT) + 2) * TR_W * 8},
      {(void**)&ws->ctrl, sizeof(Ctrl)},
  };
  for (auto& r : req) {
    cudaError_t e = cudaMalloc(r.p, r.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g3_set_error("g3_bfs workspace: cudaMalloc(%zu): %s", r.bytes, cudaGetErrorString(e));
      g3_bfs_ws_free(ws);
      return G3_ENOMEM;
    }
  }
  if (cudaMallocHost((void**)&ws->h_ctrl, sizeof(Ctrl)) != cudaSuccess) {
    cudaGetLastError();
    g3_bfs_ws_free(ws);
    return G3_ENOMEM;
  }
  for (int i = 0; i < 6; ++i)
    if (cudaEventCreate(&ws->ev[i]) != cudaSuccess) {
      cudaGetLastError();
      g3_bfs_ws_free(ws);
      return G3_ECUDA;
    }
  ws->grid_front = resident_grid(td_front, 256);
  ws->grid_bins = resident_grid(td_bins, 256);
  ws->grid_bu = resident_grid(bu_pull<1>, 256);
  int g0 = resident_grid(bu_pull<0>, 256);
  if (g0 < ws->grid_bu) ws->grid_bu = g0;
  ws->grid_conv = resident_grid(bitmap_to_q, 256);
  ws->grid_tr = resident_grid(bfs_translate, 256);
  ws->grid_trb = resident_grid(tr_bucket, 256);
  ws->grid_trw = resident_grid(tr_window, 256);
  ws->nbuckets = ((int64_t)g->n + TR_W - 1) >> TR_SHIFT;
  *out = ws;
  return G3_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static inline int cap_grid(int64_t items, int per_block, int resident) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b > resident) b = resident;
  return b < 1 ? 1 : (int)b;
}

struct Level {
  g3_graph* g;
  g3_bfs_ws* ws;
  const g3_bfs_opts* o;
  cudaStream_t s;
  uint32_t *fcur, *fnext;
  int32_t *qcur, *qnext;
  bool fmt_queue;
};

// Top-down expansion of F_L (queue qcur of length nf) into qnext. Records
// event `ev_mid` after the format conversion when given.
static g3_status run_td(Level& S, int64_t nf, int32_t lnext, cudaEvent_t ev_mid) {
  g3_bfs_ws* ws = S.ws;
  cudaStream_t s = S.s;
  if (!S.fmt_queue) {
    bitmap_to_q<<<cap_grid(ws->nwords, 256, ws->grid_conv), 256, 0, s>>>(
        S.fcur, ws->nwords, S.qcur, &ws->ctrl->conv_len);
    G3_CHECK_LAUNCH();
  }
  if (ev_mid) G3_TRY_CUDA(cudaEventRecord(ev_mid, s));
  TdArgs a{S.g->off, S.g->col, ws->visited, ws->pl, lnext, S.qnext, ws->ctrl};
  const int64_t nb1 = ws->nb + 4;
  td_front<<<cap_grid(nf, 256, ws->grid_front), 256, 0, s>>>(a, S.qcur, nf, ws->bins, ws->goff,
                                                             nb1);
  G3_CHECK_LAUNCH();
  td_bins<<<ws->grid_bins, 256, 0, s>>>(a, ws->bins, ws->goff, nb1);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

// Bottom-up expansion of F_L (bitmap) into fnext.
static g3_status run_bu(Level& S, int64_t nf, int32_t lnext, cudaEvent_t ev_mid) {
  g3_bfs_ws* ws = S.ws;
  cudaStream_t s = S.s;
  if (S.fmt_queue) {
    G3_TRY_CUDA(cudaMemsetAsync(S.fcur, 0, (size_t)ws->nwords * 4, s));
    q_to_bitmap<<<g3_grid_for(nf, 256), 256, 0, s>>>(S.qcur, nf, S.fcur);
    G3_CHECK_LAUNCH();
  }
  if (ev_mid) G3_TRY_CUDA(cudaEventRecord(ev_mid, s));
  const int grid = cap_grid(ws->nwords, 16, ws->grid_bu);
  if (S.o->bu_reverse)
    bu_pull<1><<<grid, 256, 0, s>>>(ws->nb, ws->nwords, ws->visited, S.fcur, S.fnext, S.g->off,
                                    S.g->col, ws->pl, lnext, ws->ctrl);
  else
    bu_pull<0><<<grid, 256, 0, s>>>(ws->nb, ws->nwords, ws->visited, S.fcur, S.fnext, S.g->off,
                                    S.g->col, ws->pl, lnext, ws->ctrl);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

// Candidate top-down bin thresholds timed in record_both mode.
static const int kSweep[5][3] = {
    {8, 256, 8192}, {16, 512, 16384}, {32, 1024, 32768}, {64, 2048, 65536}, {128, 4096, 131072}};

// record_both mode: time every candidate top-down expansion and the
// bottom-up one from the same state, restoring the visited bitmap and the
// controller record after each trial. Fills r (times, best thresholds); the
// state afterwards is the state before the trials.
static g3_status record_trials(Level& S, int64_t nf, int32_t L, g3_level_stats* r) {
  g3_bfs_ws* ws = S.ws;
  cudaStream_t s = S.s;
  const size_t vbytes = (size_t)ws->nwords * 4;
  G3_TRY_CUDA(cudaMemcpyAsync(ws->vis_save, ws->visited, vbytes, cudaMemcpyDeviceToDevice, s));
  Ctrl save;
  G3_TRY_CUDA(cudaMemcpyAsync(&save, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  float best = 1e30f;
  for (int k = 0; k < 6; ++k) {
    Ctrl c = save;
    const bool td = k < 5;
    if (td) {
      c.t1 = kSweep[k][0];
      c.t2 = kSweep[k][1];
      c.t3 = kSweep[k][2];
    }
    G3_TRY_CUDA(cudaMemcpyAsync(ws->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    G3_TRY_CUDA(cudaEventRecord(ws->ev[4], s));
    if (td)
      G3_TRY(run_td(S, nf, L + 1, nullptr));
    else
      G3_TRY(run_bu(S, nf, L + 1, nullptr));
    G3_TRY_CUDA(cudaEventRecord(ws->ev[5], s));
    G3_TRY_CUDA(cudaMemcpyAsync(ws->visited, ws->vis_save, vbytes, cudaMemcpyDeviceToDevice, s));
    G3_TRY_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ws->ev[4], ws->ev[5]);
    if (td && ms < best) {
      best = ms;
      r->best_t1 = kSweep[k][0];
      r->best_t2 = kSweep[k][1];
      r->best_t3 = kSweep[k][2];
    }
    if (!td) r->t_bu_ms = ms;
  }
  r->t_td_ms = best;
  G3_TRY_CUDA(cudaMemcpyAsync(ws->ctrl, &save, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  return G3_OK;
}

static g3_status bfs_impl(g3_graph* g, int32_t root, const g3_bfs_opts* o, int32_t* parent,
                          int32_t* level, g3_level_stats* stats, int32_t max_stats,
                          int32_t* n_levels, cudaStream_t s) {
  if (!g->ws) G3_TRY(ws_create(g, &g->ws));
  g3_bfs_ws* ws = g->ws;
  const int32_t nb = ws->nb;
  const int64_t nnz = g->nnz;
  Ctrl* h = ws->h_ctrl;

  G3_TRY_CUDA(cudaMemsetAsync(ws->visited, 0, (size_t)(ws->nwords + 1) * 4, s));
  bfs_root<<<1, 1, 0, s>>>(g->relabelled ? g->new_of_old : nullptr, root, nb, nnz, g->off,
                           ws->visited, ws->pl, ws->qa, ws->ctrl, o->t1, o->t2, o->t3);
  G3_CHECK_LAUNCH();

  Level S{g, ws, o, s, ws->fa, ws->fb, ws->qa, ws->qb, true};
  int nrec = 0;
  for (int32_t L = 0;; ++L) {
    G3_TRY_CUDA(cudaMemcpyAsync(h, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    G3_TRY_CUDA(cudaStreamSynchronize(s));
    if (L > 0 && stats && nrec >= 1 && nrec - 1 < max_stats) {
      // close the previous record: examined edges, next size, times
      g3_level_stats& r = stats[nrec - 1];
      r.n_next = h->nf;
      if (r.dir == G3_DIR_BU) r.examined = h->exam_prev;
      if (o->timing) {
        cudaEventElapsedTime(&r.ms, ws->ev[0], ws->ev[3]);
        cudaEventElapsedTime(&r.ms_expand, ws->ev[1], ws->ev[2]);
      }
    }
    const int64_t nf = h->nf;
    if (nf <= 0) break;
    const int dir = h->dir;
    g3_level_stats* rec = (stats && nrec < max_stats) ? &stats[nrec] : nullptr;
    if (rec) {
      memset(rec, 0, sizeof(*rec));
      rec->level = L;
      rec->dir = dir;
      rec->n_f = h->nf;
      rec->m_f = h->mf;
      rec->n_u = h->nu;
      rec->m_u = h->mu;
      rec->examined = h->mf;
      rec->id_min = h->id_min;
      rec->id_max = h->id_max;
      for (int k = 0; k < 4; ++k) rec->hist[k] = h->hist[k];
      rec->t1 = h->t1;
      rec->t2 = h->t2;
      rec->t3 = h->t3;
      for (int k = 0; k < 4; ++k) rec->mlp_out[k] = h->mlp_out[k];
    }
    ++nrec;
    if (o->record_both && rec) G3_TRY(record_trials(S, nf, L, rec));
    if (o->timing) G3_TRY_CUDA(cudaEventRecord(ws->ev[0], s));
    if (dir == G3_DIR_TD) {
      G3_TRY(run_td(S, nf, L + 1, o->timing ? ws->ev[1] : nullptr));
    } else {
      G3_TRY(run_bu(S, nf, L + 1, o->timing ? ws->ev[1] : nullptr));
    }
    if (o->timing) G3_TRY_CUDA(cudaEventRecord(ws->ev[2], s));
    bfs_control<<<1, 32, 0, s>>>(ws->ctrl, nb, nnz, o->controller, o->alpha, o->beta,
                                 o->mlp_params, o->t1, o->t2, o->t3, dir == G3_DIR_TD);
    G3_CHECK_LAUNCH();
    if (o->timing) G3_TRY_CUDA(cudaEventRecord(ws->ev[3], s));
    if (dir == G3_DIR_TD) {
      int32_t* t = S.qcur;
      S.qcur = S.qnext;
      S.qnext = t;
      S.fmt_queue = true;
    } else {
      uint32_t* t = S.fcur;
      S.fcur = S.fnext;
      S.fnext = t;
      S.fmt_queue = false;
    }
  }
  if (n_levels) *n_levels = nrec;

  // outputs in original IDs
  const bool dev_p = is_device_ptr(parent), dev_l = is_device_ptr(level);
  int32_t* op = dev_p ? parent : ws->out_parent;
  int32_t* ol = dev_l ? level : ws->out_level;
  if (g->relabelled && nrec < (1 << TR_LEVEL_BITS)) {
    G3_TRY_CUDA(cudaMemsetAsync(ws->bcount, 0, (size_t)ws->nbuckets * 4, s));
    tr_bucket<<<cap_grid(nb, 256, ws->grid_trb), 256, 0, s>>>(nb, ws->visited, ws->pl,
                                                               g->old_of_new, ws->bcount,
                                                               ws->bucket);
    G3_CHECK_LAUNCH();
    tr_window<<<cap_grid(ws->nbuckets, 1, ws->grid_trw), 256, 0, s>>>(
        g->n, root, ws->bcount, ws->bucket, op, ol);
    G3_CHECK_LAUNCH();
  } else {  // labels are the original IDs, or levels too deep for the bucket format
    bfs_translate<<<cap_grid(g->n, 256, ws->grid_tr), 256, 0, s>>>(
        g->n, nb, root, g->relabelled ? g->new_of_old : nullptr,
        g->relabelled ? g->old_of_new : nullptr, ws->visited, ws->pl, op, ol);
    G3_CHECK_LAUNCH();
  }
  if (!dev_p)
    G3_TRY_CUDA(cudaMemcpyAsync(parent, op, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
  if (!dev_l)
    G3_TRY_CUDA(cudaMemcpyAsync(level, ol, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  return G3_OK;
}

extern "C" g3_status g3_bfs(g3_graph* g, int32_t root, const g3_bfs_opts* opts, int32_t* parent,
                            int32_t* level, g3_level_stats* stats, int32_t max_stats,
                            int32_t* n_levels, void* stream) {
  if (!g || !parent || !level) {
    g3_set_error("g3_bfs: null graph or output");
    return G3_EINVAL;
  }
  if (root < 0 || root >= g->n) {
    g3_set_error("g3_bfs: root %d outside [0, %d)", root, g->n);
    return G3_EINVAL;
  }
  g3_bfs_opts o;
  if (opts) o = *opts; else g3_bfs_opts_default(&o);
  if (o.controller < 0 || o.controller > 3 || o.alpha <= 0 || o.beta <= 0 || o.t1 < 1 ||
      o.t2 <= o.t1 || o.t3 <= o.t2) {
    g3_set_error("g3_bfs: bad options");
    return G3_EINVAL;
  }
  if (o.controller == G3_CTRL_LEARNED && !o.mlp_params) {
    g3_set_error("g3_bfs: learned controller needs mlp_params");
    return G3_EINVAL;
  }
  if (max_stats < 0) max_stats = 0;
  cudaStream_t s = (cudaStream_t)stream;
  g3_status st = bfs_impl(g, root, &o, parent, level, stats, max_stats, n_levels, s);
  if (st != G3_OK) cudaStreamSynchronize(s);
  return st;
}
