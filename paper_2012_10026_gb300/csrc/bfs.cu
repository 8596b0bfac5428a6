// Hybrid breadth-first search (Algorithm 2) on the graph's current CSR.
//
// Per level L the frontier F_L is either a queue (after a top-down level) or
// a bitmap (after a bottom-up level). A one-warp controller kernel decides
// the direction of every level on the device from the frontier statistics
// and records which buffers hold the frontier; every expansion kernel reads
// its direction, sizes and buffers from that device-side record. So the whole
// level loop can run without the host:
//
//   graph mode (default): one CUDA graph per search -- a WHILE node whose body
//     is a SWITCH over the four level kinds {top-down from a queue, top-down
//     from a bitmap, bottom-up from a bitmap, bottom-up from a queue} followed
//     by the controller, which sets the next kind and ends the loop. A launch
//     runs at most GRAPH_LEVEL_CAP levels; deeper searches continue on the
//     host-driven path from the same state.
//   host-driven mode (per-level timing or record_both): the host reads the
//     controller record after every level and launches the same kernels.
//
//   top-down (Algorithms 1 and 4): td_front walks the queue one thread per
//     vertex; vertices with degree < t1 are expanded on the spot, the others
//     go to three bins: one warp (t1 <= deg < t2), one CTA (t2 <= deg < t3)
//     or the grid bin (deg >= t3), whose lists are flattened into one edge
//     range split evenly over all warps -- the GPU form of Algorithm 4's even
//     split. Neighbour lists are read with aligned 128-bit loads. A neighbour
//     is claimed by an atomicOr on its word of the visited bitmap; the winner
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
// per block; the controller logs them per level. (parent, level) of BFS-graph
// vertices are kept packed as int2 and are only meaningful where the visited
// bit is set, so nothing but the visited bitmap is cleared per search. The
// outputs in original IDs are then gathered in one pass (bfs_translate4).
#include <math.h>
#include <string.h>

#include "g3_mlp.cuh"
#include "g3_prims.cuh"

#define LOG_MAX 4096           // per-level records kept on the device
#define GRAPH_LEVEL_CAP 4096   // levels one graph launch may run

// Level kinds (the SWITCH branch a level runs): top-down from a queue or a
// bitmap frontier, bottom-up from a bitmap or a queue frontier, the same on
// a sparse level (vertex list, see bu_list_build), and the end.
enum {
  MODE_TD_Q = 0, MODE_TD_B = 1, MODE_BU_B = 2, MODE_BU_Q = 3, MODE_DONE = 4,
  MODE_BU_BS = 5, MODE_BU_QS = 6, MODE_TD_QS = 7, MODE_COUNT = 8
};
// A top-down level from a queue this small (frontier vertices, their edges)
// runs the same kernels on TD_SMALL_GRID blocks: launching and retiring a
// grid sized for the largest levels costs more than such a level's work.
#define TD_SMALL_NF 16384
#define TD_SMALL_MF 65536
#define TD_SMALL_GRID 64

// Device-side controller record.
struct __align__(16) Ctrl {
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
  long long nf, mf, nu, mu;
  long long hist[4];
  int id_min, id_max;
  int level;
  int dir;
  int t1, t2, t3;
  float mlp_out[4];
  long long n_visited, m_visited;
  // where F_L lives: fmt_queue 0 bitmap f[fsel], 1 queue q[qsel], 2 both
  // (a sparse bottom-up level writes its next frontier in both forms)
  int qsel, fsel, fmt_queue;
  int mode;  // MODE_* of the current level
  int cap;   // the controller ends the search at this level (graph launches)
  unsigned int err;  // a kernel's bounded wait ran out (the search stops; G3_ETIMEOUT)
  int full_stats;    // keep the degree histogram and label range of each frontier
  // rng_ok: the search reaches exactly the labels [rng_lo, rng_hi), the root's
  // component (known after a full RCM relabel); else the visited bitmap tells
  int rng_ok, rng_lo, rng_hi;
  int bu_sparse;                  // this bottom-up level runs over a vertex list
  unsigned long long bl_len;      // that list's length
};

// Per-level record written by the controller (and bfs_root for level 0).
struct LevelLog {
  int dir, t1, t2, t3;
  long long nf, mf, nu, mu, examined, n_next;
  int id_min, id_max;
  long long hist[4];
  float mlp_out[4];
};

struct Bufs {
  int32_t* q[2];
  uint32_t* f[2];
  const int32_t* o2n;  // old_of_new (parents are stored as original IDs), or NULL
};

// (parent's original ID, level) of a labelled vertex packed into one 32-bit
// word, parent << bits | min(level, lmax) with lmax = 2^bits - 1 and bits =
// 32 - (bits of n - 1); a level >= lmax is also kept in deep[x]. At SCALE 26
// the word holds levels up to 62 by itself, and the packed array (4 B per
// vertex) is half the size the output pass has to gather from.
struct PlOut {
  uint32_t* pl;
  int32_t* deep;
  int32_t bits;
};

// The packed words are stored with an L2 evict-last policy: the output pass
// gathers them after the search, so they should outlive the streamed rows.
__device__ __forceinline__ void st_keep_l2(uint32_t* a, uint32_t v) {
  uint64_t pol;  // a constant: not volatile, so the compiler creates it once
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol)
               : "memory");
}

__device__ __forceinline__ void pl_put(const PlOut& o, int32_t x, int32_t parent,
                                       int32_t level) {
  const uint32_t lmax = (1u << o.bits) - 1u;
  const uint32_t code = (uint32_t)level < lmax ? (uint32_t)level : lmax;
  st_keep_l2(o.pl + x, ((uint32_t)parent << o.bits) | code);
  if ((uint32_t)level >= lmax) o.deep[x] = level;
}

__device__ __forceinline__ int2 pl_decode(const PlOut& o, uint32_t w, int32_t x) {
  const uint32_t lmax = (1u << o.bits) - 1u;
  const uint32_t code = w & lmax;
  return make_int2((int32_t)(w >> o.bits), code == lmax ? __ldg(&o.deep[x]) : (int32_t)code);
}

static int32_t pl_bits(int32_t n) {
  int bp = 1;
  while (bp < 31 && ((int64_t)1 << bp) < (int64_t)n) ++bp;
  return 32 - bp;
}

struct g3_bfs_ws {
  int32_t nb;
  int64_t nwords;
  uint32_t *visited, *fa, *fb, *vis_save;
  int32_t *qa, *qb, *bins;  // bins: 3 segments of nb entries (warp, CTA, grid)
  int64_t* goff;            // edge offset of each grid-bin vertex
  PlOut plo;                // packed (parent, level) per BFS-graph vertex
  int2* nplus;              // (last row entry or -1, degree): Algorithm 6's neighbors+
  int32_t *out_parent, *out_level;  // staging for host outputs (n entries)
  Ctrl* ctrl;
  Ctrl* h_ctrl;  // pinned
  LevelLog* log;
  cudaEvent_t ev[6];
  // resident-grid sizes (SMs x blocks per SM) per kernel
  int grid_front, grid_bins, grid_bu, grid_tiles, grid_staged, grid_conv, grid_tr, grid_tr4;
  int grid_lb, grid_lp;  // sparse bottom-up: list build, list pull
  // graph mode: instantiated level loop and the options it was built for
  cudaGraphExec_t gexec;
  g3_bfs_opts gopts;
  int gfull;  // the statistics mode the cached graph's kernels were built for
};

void g3_bfs_ws_free(g3_bfs_ws* ws) {
  if (!ws) return;
  void* all[] = {ws->visited,    ws->fa,        ws->fb,   ws->vis_save, ws->qa,
                 ws->qb,         ws->bins,      ws->plo.pl, ws->plo.deep, ws->out_parent,
                 ws->out_level,  ws->ctrl,      ws->goff, ws->nplus,
                 ws->log};
  for (void* p : all)
    if (p) cudaFree(p);
  if (ws->h_ctrl) cudaFreeHost(ws->h_ctrl);
  for (int i = 0; i < 6; ++i)
    if (ws->ev[i]) cudaEventDestroy(ws->ev[i]);
  if (ws->gexec) cudaGraphExecDestroy(ws->gexec);
  free(ws);
}

// ----------------------------------------------------------- device helpers
__device__ __forceinline__ int deg_bucket(int64_t d) {
  return d < 32 ? 0 : (d < 1024 ? 1 : (d < 32768 ? 2 : 3));
}

// Per-thread statistics in 32-bit registers (a thread sees far fewer than
// 2^32 vertices or edges per launch); reduced per block in 64 bits.
// The degree histogram and the label range are kept only when the search
// records its per-level statistics (Ctrl::full_stats); both controllers need
// only sizes and degree sums. MODE 0 keeps sizes and sums only, 1 everything,
// 2 decides at run time from Ctrl::full_stats (a kernel instantiated for
// MODE 0 or 1 is launched only when that matches).
template <int MODE>
struct StatAccT {
  unsigned nf, mf, ex, h0, h1, h2, h3, mn, mx;
  bool full;
  __device__ void init(const Ctrl* c) {
    nf = mf = ex = h0 = h1 = h2 = h3 = 0;
    mn = 0xFFFFFFFFu;
    mx = 0;
    full = MODE == 2 ? c->full_stats != 0 : MODE == 1;
  }
  __device__ void add_vertex(int32_t v, int64_t d) {
    nf++;
    mf += (unsigned)d;
    if (MODE == 0 || !full) return;
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
    const int nk = MODE == 0 ? 3 : 7;
    unsigned long long v[7] = {nf, mf, ex, h0, h1, h2, h3};
    unsigned a = mn, b = mx;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
      for (int k = 0; k < nk; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      if (MODE != 0) {
        a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
      }
    }
    if (lane == 0) {
      for (int k = 0; k < nk; ++k) s[warp][k] = v[k];
      smn[warp] = a;
      smx[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t[7] = {0, 0, 0, 0, 0, 0, 0};
      unsigned tmn = 0xFFFFFFFFu, tmx = 0;
      for (int w = 0; w < nw; ++w) {
        for (int k = 0; k < nk; ++k) t[k] += s[w][k];
        tmn = min(tmn, smn[w]);
        tmx = max(tmx, smx[w]);
      }
      if (t[0]) atomicAdd(&c->nx_nf, t[0]);
      if (t[1]) atomicAdd(&c->nx_mf, t[1]);
      if (t[2]) atomicAdd(&c->nx_exam, t[2]);
      if (MODE == 0) return;
      for (int k = 0; k < 4; ++k)
        if (t[3 + k]) atomicAdd(&c->nx_hist[k], t[3 + k]);
      if (t[0]) {
        atomicMin(&c->nx_min, tmn);
        atomicMax(&c->nx_max, tmx);
      }
    }
  }
};
using StatAcc = StatAccT<2>;

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
  c->bl_len = 0;
}

__device__ __forceinline__ int mode_of(const Ctrl* c) {
  if (c->nf <= 0) return MODE_DONE;
  if (c->dir == G3_DIR_TD) {
    if (!c->fmt_queue) return MODE_TD_B;
    return c->nf <= TD_SMALL_NF && c->mf <= TD_SMALL_MF ? MODE_TD_QS : MODE_TD_Q;
  }
  const bool only_queue = c->fmt_queue == 1;
  if (c->bu_sparse) return only_queue ? MODE_BU_QS : MODE_BU_BS;
  return only_queue ? MODE_BU_Q : MODE_BU_B;
}

// A bottom-up level with under 4 % of the graph unvisited runs over a list
// of its unvisited vertices (bu_kernel 0); above that the word-pair kernel's
// coalesced walk is the faster one (measured on Kronecker graphs).
#ifndef BU_LIST_PM
#define BU_LIST_PM 40
#endif
__host__ __device__ __forceinline__ bool bu_sparse_level(long long nu, int32_t nb) {
  return nu * 1000 < (long long)nb * BU_LIST_PM;
}

__device__ __forceinline__ void log_frontier(LevelLog* log, const Ctrl* c) {
  if (c->level >= LOG_MAX) return;
  LevelLog& r = log[c->level];
  r.dir = c->dir;
  r.t1 = c->t1;
  r.t2 = c->t2;
  r.t3 = c->t3;
  r.nf = c->nf;
  r.mf = c->mf;
  r.nu = c->nu;
  r.mu = c->mu;
  r.examined = c->mf;
  r.n_next = 0;
  r.id_min = c->id_min;
  r.id_max = c->id_max;
  for (int k = 0; k < 4; ++k) {
    r.hist[k] = c->hist[k];
    r.mlp_out[k] = c->mlp_out[k];
  }
}

// ------------------------------------------------------------------- init
// Sets up F_0 = {root} (root_new < 0 or >= nb: no BFS-graph vertex). The
// visited bitmap has been cleared on the stream before. comp (nullable): the
// label range of each label's component.
__global__ void bfs_root(const int32_t* new_of_old, const int2* comp, int32_t root, int32_t nb,
                         int64_t nnz, const int64_t* off, uint32_t* visited, PlOut plo,
                         int32_t* q, Ctrl* c, LevelLog* log, int t1, int t2, int t3, int cap,
                         int full_stats) {
  int32_t r = new_of_old ? new_of_old[root] : root;
  memset(c, 0, sizeof(Ctrl));
  reset_next(c);
  if (comp) {  // an isolated root reaches no label: the empty range
    const int2 cr = (r >= 0 && r < nb) ? comp[r] : make_int2(0, 0);
    c->rng_ok = 1;
    c->rng_lo = cr.x;
    c->rng_hi = cr.y;
  }
  c->full_stats = full_stats;
  c->t1 = t1;
  c->t2 = t2;
  c->t3 = t3;
  c->dir = G3_DIR_TD;  // Algorithm 2 starts top-down
  c->fmt_queue = 1;
  c->cap = cap;
  if (r < 0 || r >= nb) {
    c->nf = 0;
    c->nu = nb;
    c->mu = nnz;
    c->mode = MODE_DONE;
    return;
  }
  visited[r >> 5] |= 1u << (r & 31);
  pl_put(plo, r, root, 0);  // parents are kept as original IDs
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
  c->mode = MODE_TD_Q;
  log_frontier(log, c);
}

// Sets up F_0 with several roots at once: root i counts when it is a
// BFS-graph vertex and, with lo given, lies in [lo[i], lo[i+1]) (the batched
// search over disjoint graphs seeds one root per graph, so their levels
// cannot interfere). Repeated roots are seeded once. One block.
__global__ void __launch_bounds__(1024) bfs_roots_multi(
    const int32_t* __restrict__ roots, int32_t count, const int32_t* __restrict__ lo,
    const int32_t* new_of_old, int32_t nb, int64_t nnz, const int64_t* off, uint32_t* visited,
    PlOut plo, int32_t* q, Ctrl* c, LevelLog* log, int t1, int t2, int t3, int cap,
    int full_stats) {
  __shared__ unsigned long long s_nf, s_mf, s_hist[4];
  __shared__ int s_min, s_max;
  if (threadIdx.x == 0) {
    s_nf = s_mf = 0;
    for (int k = 0; k < 4; ++k) s_hist[k] = 0;
    s_min = 0x7fffffff;
    s_max = -1;
  }
  __syncthreads();
  for (int32_t i = threadIdx.x; i < count; i += blockDim.x) {
    const int32_t root = roots[i];
    if (lo && (root < lo[i] || root >= lo[i + 1])) continue;
    const int32_t r = new_of_old ? new_of_old[root] : root;
    if (r < 0 || r >= nb) continue;
    const uint32_t bit = 1u << (r & 31);
    if (atomicOr(&visited[r >> 5], bit) & bit) continue;
    pl_put(plo, r, root, 0);
    q[atomicAdd(&s_nf, 1ull)] = r;
    const long long d = off[r + 1] - off[r];
    atomicAdd(&s_mf, (unsigned long long)d);
    atomicAdd(&s_hist[deg_bucket(d)], 1ull);
    atomicMin(&s_min, r);
    atomicMax(&s_max, r);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  memset(c, 0, sizeof(Ctrl));
  reset_next(c);
  c->full_stats = full_stats;
  c->t1 = t1;
  c->t2 = t2;
  c->t3 = t3;
  c->dir = G3_DIR_TD;
  c->fmt_queue = 1;
  c->cap = cap;
  const long long nf = (long long)s_nf, mf = (long long)s_mf;
  if (nf == 0) {
    c->nu = nb;
    c->mu = nnz;
    c->mode = MODE_DONE;
    return;
  }
  c->nf = nf;
  c->mf = mf;
  for (int k = 0; k < 4; ++k) c->hist[k] = (long long)s_hist[k];
  c->id_min = s_min;
  c->id_max = s_max;
  c->n_visited = nf;
  c->m_visited = mf;
  c->nu = nb - nf;
  c->mu = nnz - mf;
  c->mode = MODE_TD_Q;
  log_frontier(log, c);
}

// --------------------------------------------------------------- top-down
struct TdArgs {
  const int64_t* off;
  const int32_t* col;
  uint32_t* visited;
  PlOut plo;
  int32_t lnext;
  int32_t* qnext;
  Ctrl* c;
  const int32_t* o2n;
};

__device__ __forceinline__ int32_t orig_of(const int32_t* o2n, int32_t v) {
  return o2n ? __ldg(&o2n[v]) : v;
}

// Per-warp staging of the next queue in shared memory: claimed vertices are
// compacted into the warp's buffer with ballots and written to the global
// queue in one coalesced burst, reserving space with one atomic per few
// hundred vertices instead of one per warp step (the queue counter is a
// single address that every warp of the grid would otherwise hit). The
// statistics of the claimed vertices (degree sum, histogram, label range)
// are taken at flush time, when the lanes load the degrees of up to 16
// staged vertices each at once, instead of inside each claim's dependent
// chain.
#define WQ_CAP 512
#define WQ_FLUSH (WQ_CAP - 128)
struct WarpQueue {
  int32_t* buf;  // this warp's WQ_CAP-entry shared buffer
  int cnt;       // warp-uniform fill level
};

__device__ __forceinline__ void wq_flush(WarpQueue& q, const TdArgs& a, StatAcc& acc) {
  if (q.cnt == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&a.c->q_len, (unsigned long long)q.cnt);
  base = __shfl_sync(0xffffffffu, base, 0);
  __syncwarp();
  for (int k0 = 0; k0 < q.cnt; k0 += 256) {  // eight entries per lane at a time
    int32_t w[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = k0 + lane + 32 * k;
      w[k] = i < q.cnt ? q.buf[i] : -1;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = w[k] >= 0 ? (int32_t)(a.off[w[k] + 1] - a.off[w[k]]) : 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (w[k] >= 0) {
        a.qnext[base + k0 + lane + 32 * k] = w[k];
        acc.add_vertex(w[k], d[k]);
      }
  }
  __syncwarp();
  q.cnt = 0;
}

// Appends up to four items per lane (want[k]); all 32 lanes call it together.
__device__ __forceinline__ void wq_push4(WarpQueue& q, const bool want[4], const int32_t item[4],
                                         const TdArgs& a, StatAcc& acc) {
  // most steps claim nothing (the visited probe already saw the bit set)
  if (!__any_sync(0xffffffffu, want[0] | want[1] | want[2] | want[3])) return;
  const unsigned lt = g3_lanemask_lt();
  int at = q.cnt;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned bal = __ballot_sync(0xffffffffu, want[k]);
    if (want[k]) q.buf[at + __popc(bal & lt)] = item[k];
    at += __popc(bal);
  }
  if (at == q.cnt) return;
  q.cnt = at;
  __syncwarp();
  if (q.cnt > WQ_FLUSH) wq_flush(q, a, acc);
}

#define WQ_DECLARE(q)                                      \
  __shared__ int32_t wq_mem[8][WQ_CAP];                    \
  WarpQueue q{wq_mem[threadIdx.x >> 5], 0}

// Claims up to four neighbours w[k] (has[k]) for v at once: the four
// visited-word reads, then the atomicOr of those still clear, are issued
// together so that a lane keeps four claims in flight instead of one
// dependent read-atomic pair at a time. The winners write (parent, level)
// and are appended to the next queue. All 32 lanes must call it together.
__device__ __forceinline__ void td_visit4(const TdArgs& a, WarpQueue& q, StatAcc& acc,
                                          const bool has[4], const int32_t w[4], int32_t v) {
  uint32_t word[4];
  bool cand[4];
#pragma unroll
  // the probes may hit L1: during a level bits only turn from 0 to 1, so a
  // stale word can only say "unvisited", and the atomicOr then tells the truth
  for (int k = 0; k < 4; ++k) word[k] = has[k] ? __ldca(&a.visited[w[k] >> 5]) : ~0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) cand[k] = has[k] && !((word[k] >> (w[k] & 31)) & 1u);
  uint32_t old[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    old[k] = cand[k] ? atomicOr(&a.visited[w[k] >> 5], 1u << (w[k] & 31)) : ~0u;
  bool claim[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) claim[k] = cand[k] && !((old[k] >> (w[k] & 31)) & 1u);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (claim[k]) pl_put(a.plo, w[k], v, a.lnext);  // v: the parent's original ID
  wq_push4(q, claim, w, a, acc);
}

// Processes row entries [b, e) of vertex v with `nthr` cooperating threads
// (index t), four entries per thread per step through aligned 128-bit loads.
// Every lane of each participating warp runs the same number of steps.
__device__ __forceinline__ void td_row_vec4(const TdArgs& a, WarpQueue& q, StatAcc& acc,
                                            int32_t v, int64_t b, int64_t e, int64_t t,
                                            int64_t nthr, int64_t steps) {
  const int64_t a0 = b & ~3ll;
  const int32_t vo = orig_of(a.o2n, v);
  // the next step's entries are loaded before this step's claims, so the
  // row read overlaps the visited probes and atomics instead of preceding them
  int64_t j = a0 + 4 * t;
  int4 x = make_int4(0, 0, 0, 0);
  if (steps > 0 && j < e) x = *reinterpret_cast<const int4*>(a.col + j);
  for (int64_t s = 0; s < steps; ++s) {
    const int64_t jn = j + 4 * nthr;
    int4 xn = make_int4(0, 0, 0, 0);
    if (s + 1 < steps && jn < e) xn = *reinterpret_cast<const int4*>(a.col + jn);
    bool has[4];
    if (j >= b && j + 3 < e) {  // an interior step: all four entries
      has[0] = has[1] = has[2] = has[3] = true;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) has[k] = j + k >= b && j + k < e;
    }
    const int32_t w[4] = {x.x, x.y, x.z, x.w};
    td_visit4(a, q, acc, has, w, vo);
    j = jn;
    x = xn;
  }
}

// Grid-bin slots and their edge offsets are handed out by one 64-bit atomic
// (slot count in the high bits, edge total in the low 38 bits), so the offsets
// ascend with the slot index.
#define GP_SHIFT 38
#define GP_MASK ((1ull << GP_SHIFT) - 1ull)

__device__ __forceinline__ TdArgs td_args(const int64_t* off, const int32_t* col,
                                          uint32_t* visited, const PlOut& plo, const Bufs& B,
                                          Ctrl* c) {
  return TdArgs{off, col, visited, plo, c->level + 1, (c->qsel ? B.q[0] : B.q[1]), c, B.o2n};
}

// Thread per frontier vertex: degree < t1 expanded here, larger degrees
// binned (warp / CTA / grid).
__global__ void __launch_bounds__(256) td_front(const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ col,
                                                uint32_t* visited, PlOut plo, Bufs B,
                                                int32_t* bins, int64_t* goff, int64_t nb1,
                                                Ctrl* c) {
  if (c->dir != G3_DIR_TD) return;
  const TdArgs a = td_args(off, col, visited, plo, B, c);
  const int32_t* __restrict__ q = (c->qsel ? B.q[1] : B.q[0]);
  const int64_t qlen = c->nf;
  const int t1 = c->t1, t2 = c->t2, t3 = c->t3;
  WQ_DECLARE(wq);
  StatAcc acc;
  acc.init(c);
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < qlen;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool act = i < qlen;
    int32_t v = act ? q[i] : 0;
    int64_t b = act ? off[v] : 0, e = act ? off[v + 1] : 0, d = e - b;
    bool small = act && d < t1;
    int bin = !act || small ? -1 : (d < t2 ? 0 : (d < t3 ? 1 : 2));
    for (int k = 0; k < 2; ++k)
      g3_warp_append(0xffffffffu, bin == k, v, bins + k * nb1, &c->bin_len[1 + k]);
    if (bin == 2) {
      const unsigned long long old =
          atomicAdd(&c->g_pack, (1ull << GP_SHIFT) | (unsigned long long)d);
      const int64_t slot = (int64_t)(old >> GP_SHIFT);
      bins[2 * nb1 + slot] = v;
      goff[slot] = (int64_t)(old & GP_MASK);
    }
    const int cnt = small ? (int)d : 0;
    const int maxc = __reduce_max_sync(0xffffffffu, cnt);
    const int32_t vo = cnt ? orig_of(a.o2n, v) : 0;
    for (int k = 0; k < maxc; k += 4) {
      bool has[4];
      int32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        has[u] = k + u < cnt;
        w[u] = has[u] ? col[b + k + u] : 0;
      }
      td_visit4(a, wq, acc, has, w, vo);
    }
  }
  wq_flush(wq, a, acc);
  acc.flush(c);
}

// The three bins in one launch: warp per warp-bin vertex, CTA per CTA-bin
// vertex, and the grid bin as one flattened edge range split evenly over all
// warps of the grid (Algorithm 4's even split, applied to every hub at once).
__global__ void __launch_bounds__(256, 4) td_bins(const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ col,
                                               uint32_t* visited, PlOut plo, Bufs B,
                                               const int32_t* __restrict__ bins,
                                               const int64_t* __restrict__ goff, int64_t nb1,
                                               Ctrl* c) {
  if (c->dir != G3_DIR_TD) return;
  const TdArgs a = td_args(off, col, visited, plo, B, c);
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  WQ_DECLARE(wq);
  StatAcc acc;
  acc.init(c);
  const int64_t len1 = (int64_t)c->bin_len[1];
  for (int64_t i = gw; i < len1; i += nwarps) {
    int32_t v = bins[i];
    int64_t b = off[v], e = off[v + 1];
    int64_t steps = (e - (b & ~3ll) + 127) / 128;
    td_row_vec4(a, wq, acc, v, b, e, lane, 32, steps);
  }
  const int64_t len2 = (int64_t)c->bin_len[2];
  for (int64_t i = blockIdx.x; i < len2; i += gridDim.x) {
    int32_t v = bins[nb1 + i];
    int64_t b = off[v], e = off[v + 1];
    int64_t steps = (e - (b & ~3ll) + 4 * blockDim.x - 1) / (4 * blockDim.x);
    td_row_vec4(a, wq, acc, v, b, e, threadIdx.x, blockDim.x, steps);
  }
  const unsigned long long gp = c->g_pack;
  const int64_t nh = (int64_t)(gp >> GP_SHIFT), E = (int64_t)(gp & GP_MASK);
  if (E > 0) {
    // every warp owns an equal range [j0, j1) of the hubs' concatenated
    // lists and walks the hub segments it overlaps, 128 entries per step
    const int32_t* gbin = bins + 2 * nb1;
    const int64_t per = (((E + nwarps - 1) / nwarps) + 127) & ~127ll;
    const int64_t j0 = gw * per, j1 = min(E, j0 + per);
    if (j0 < j1) {
      for (int64_t h = g3_upper_bound_i64(goff, nh, j0) - 1; h < nh && goff[h] < j1; ++h) {
        const int64_t s0 = max(j0, goff[h]);
        const int64_t s1 = min(j1, h + 1 < nh ? goff[h + 1] : E);
        if (s0 >= s1) continue;
        const int32_t v = gbin[h];
        const int64_t rb = off[v] + (s0 - goff[h]), re = off[v] + (s1 - goff[h]);
        const int64_t steps = (re - (rb & ~3ll) + 127) / 128;
        td_row_vec4(a, wq, acc, v, rb, re, lane, 32, steps);
      }
    }
  }
  wq_flush(wq, a, acc);
  acc.flush(c);
}

// -------------------------------------------------------------- bottom-up
// Where two bottom-up kernels share a level kind (bu_kernel 1: staged and
// word tiles; 3: word pairs and word tiles), levels with at least a quarter
// of the graph unvisited are the first kernel's and the others the word-tile
// kernel's; both check this same condition. (bu_kernel 0 splits the levels
// by bu_sparse_level instead, in the controller.)
__device__ __forceinline__ bool bu_dense(const Ctrl* c, int32_t nb) {
  return c->nu * 4 >= (long long)nb;
}

__device__ __forceinline__ bool in_frontier(const uint32_t* __restrict__ f, int32_t w) {
  return (__ldg(&f[w >> 5]) >> (w & 31)) & 1u;
}

// Scans the rest of a row after a missed first probe; returns the parent or
// -1 and advances k (edges examined, up to and including the parent, as a
// one-at-a-time scan counts them). Four entries per step: their column
// loads, then their frontier probes, are in flight together, so a row of a
// few entries costs one dependent round trip instead of one per entry (on a
// dense level most of the time goes into these scans). Entries past the
// row's end are never loaded.
template <int REV>
__device__ __forceinline__ int32_t bu_scan_rest(const int32_t* __restrict__ col,
                                                const uint32_t* __restrict__ fcur, int64_t b,
                                                int64_t e, int64_t& k) {
  const int64_t d = e - b;
  const int32_t* __restrict__ p = REV ? col + (e - 1) : col + b;  // entry k at p[+-k]
  const int64_t step = REV ? -1 : 1;
  while (k < d) {
    const int64_t left = d - k;
    const int32_t w0 = __ldg(p + step * k);
    const int32_t w1 = left > 1 ? __ldg(p + step * (k + 1)) : 0;
    const int32_t w2 = left > 2 ? __ldg(p + step * (k + 2)) : 0;
    const int32_t w3 = left > 3 ? __ldg(p + step * (k + 3)) : 0;
    const bool f0 = in_frontier(fcur, w0);
    const bool f1 = left > 1 && in_frontier(fcur, w1);
    const bool f2 = left > 2 && in_frontier(fcur, w2);
    const bool f3 = left > 3 && in_frontier(fcur, w3);
    if (f0) { k += 1; return w0; }
    if (f1) { k += 2; return w1; }
    if (f2) { k += 3; return w2; }
    if (f3) { k += 4; return w3; }
    k += left < 4 ? left : 4;
  }
  return -1;
}

// Rest of a row after a missed first probe, four entries per step: their
// four column loads and then their four frontier probes are in flight
// together, and the first hit in scan order wins, so k (entries examined, up
// to and including the parent) is the same as for a one-at-a-time scan.
// Entries past the row's end are never loaded.
template <int REV>
__device__ __forceinline__ int32_t bu_scan_rest4(const int32_t* __restrict__ col,
                                                 const uint32_t* __restrict__ fcur, int64_t b,
                                                 int64_t e, int64_t& k) {
  const int64_t d = e - b;
  while (k < d) {
    int32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t kk = k + q;
      w[q] = kk < d ? __ldg(&col[REV ? e - 1 - kk : b + kk]) : -1;
    }
    bool h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = w[q] >= 0 && in_frontier(fcur, w[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (h[q]) {
        k += q + 1;
        return w[q];
      }
    k = k + 4 < d ? k + 4 : d;
  }
  return -1;
}

// Bottom-up level over word pairs (Algorithms 5 and 6): a warp owns two
// consecutive words of the visited bitmap per grid step and lane i the
// vertex of bit i of each, so the neighbors+ loads of a warp are coalesced,
// and two vertices per lane are in flight. FULL: the per-level histogram and
// label range are kept too (a separate instantiation, so that the default
// one carries only the counters the controllers read).
template <int REV, int FULL>
__global__ void __launch_bounds__(256, 8) bu_pull(int32_t nb, int64_t nwords, uint32_t* visited,
                                               Bufs B, const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ col,
                                               const int2* __restrict__ nplus, PlOut plo,
                                               Ctrl* c, int sparse_to_tiles) {
  // sparse_to_tiles: levels with under a quarter of the graph unvisited are
  // left to the word-tile kernel launched beside this one
  if (c->dir != G3_DIR_BU || (sparse_to_tiles && !bu_dense(c, nb))) return;
  const uint32_t* __restrict__ fcur = (c->fsel ? B.f[1] : B.f[0]);
  uint32_t* __restrict__ fnext = (c->fsel ? B.f[0] : B.f[1]);
  const int32_t lnext = c->level + 1;
  const int32_t* __restrict__ o2n = B.o2n;
  StatAccT<FULL> acc;
  acc.init(c);
  const int lane = threadIdx.x & 31;
  // word and vertex indices fit 32 bits (nb < 2^31); row offsets stay 64-bit
  const int32_t nw = (int32_t)nwords;
  const int32_t nwarps = (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5);
  const int32_t wid = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  for (int32_t w0 = 2 * wid; w0 < nw; w0 += 2 * nwarps) {
    const bool has1 = w0 + 1 < nw;
    const uint32_t vis0 = visited[w0];
    const uint32_t vis1 = has1 ? visited[w0 + 1] : 0xFFFFFFFFu;
    const int32_t v0 = w0 * 32 + lane, v1 = v0 + 32;
    const bool c0 = v0 < nb && !((vis0 >> lane) & 1u);
    const bool c1 = v1 < nb && !((vis1 >> lane) & 1u);
    if (!__any_sync(0xffffffffu, c0 || c1)) {
      if (lane == 0) {
        fnext[w0] = 0u;
        if (has1) fnext[w0 + 1] = 0u;
      }
      continue;
    }
    // first probes of both vertices, independent of each other. In the
    // degree-aware order the first candidate is the row's last entry, read
    // from the dense neighbors+ array together with the degree (8 coalesced
    // bytes per vertex instead of two row bounds and a 32-byte sector).
    int64_t b0 = 0, e0 = 0, b1 = 0, e1 = 0;
    int32_t x0 = -1, x1 = -1, d0 = 0, d1 = 0;
    if (REV) {
      if (c0) {
        const int2 t = nplus[v0];
        x0 = t.x;
        d0 = t.y;
      }
      if (c1) {
        const int2 t = nplus[v1];
        x1 = t.x;
        d1 = t.y;
      }
    } else {
      if (c0) {
        b0 = off[v0];
        e0 = off[v0 + 1];
        d0 = (int32_t)(e0 - b0);
        if (d0) x0 = col[b0];
      }
      if (c1) {
        b1 = off[v1];
        e1 = off[v1 + 1];
        d1 = (int32_t)(e1 - b1);
        if (d1) x1 = col[b1];
      }
    }
    int32_t p0 = (x0 >= 0 && in_frontier(fcur, x0)) ? x0 : -1;
    int32_t p1 = (x1 >= 0 && in_frontier(fcur, x1)) ? x1 : -1;
    int64_t k0 = d0 > 0 ? 1 : 0, k1 = d1 > 0 ? 1 : 0;
    const bool m0 = p0 < 0 && d0 > 1, m1 = p1 < 0 && d1 > 1;
    if (REV) {  // the first probe came from neighbors+: the row bounds now
      if (m0) {
        e0 = off[v0 + 1];
        b0 = e0 - d0;
      }
      if (m1) {
        e1 = off[v1 + 1];
        b1 = e1 - d1;
      }
    }
    // (a warp-wide scan of the long rows was slower: under RCM the long rows
    // come clustered, and one lane per row keeps them all in flight)
    if (m0) p0 = bu_scan_rest<REV>(col, fcur, b0, e0, k0);
    if (m1) p1 = bu_scan_rest<REV>(col, fcur, b1, e1, k1);
    acc.ex += (unsigned)(k0 + k1);
    const int32_t q0 = p0 >= 0 && o2n ? __ldg(&o2n[p0]) : p0;
    const int32_t q1 = p1 >= 0 && o2n ? __ldg(&o2n[p1]) : p1;
    const uint32_t n0 = __ballot_sync(0xffffffffu, p0 >= 0);
    const uint32_t n1 = __ballot_sync(0xffffffffu, p1 >= 0);
    if (p0 >= 0) {
      pl_put(plo, v0, q0, lnext);
      acc.add_vertex(v0, d0);
    }
    if (p1 >= 0) {
      pl_put(plo, v1, q1, lnext);
      acc.add_vertex(v1, d1);
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

// Bottom-up on a sparse level (Algorithm 6's shrinking of the active range,
// taken down to single vertices). Walking the bitmap two words per warp step
// costs a load latency per step even where every vertex is visited, which
// dominates a level with a few thousand unvisited vertices in a million
// words. Instead bu_list_build lists the unvisited vertices (a lane per
// word, one atomic per warp to place its slice) and clears the next-frontier
// words, and bu_list_pull gives every listed vertex its own thread, all in
// flight at once; a found vertex sets its bits in the next frontier and the
// visited bitmap with atomic ORs and is also appended to a queue, so that a
// top-down level after this one needs no bitmap -> queue pass. The list goes
// into the queue that is not the current frontier, the found vertices into
// the other one (whose frontier, if it had one, the bitmap already holds).
__global__ void __launch_bounds__(256) bu_list_build(Bufs B, int64_t nwords, int32_t nb,
                                                     const uint32_t* __restrict__ visited,
                                                     Ctrl* c) {
  if (c->dir != G3_DIR_BU) return;
  uint32_t* __restrict__ fnext = (c->fsel ? B.f[0] : B.f[1]);
  int32_t* __restrict__ list = (c->qsel ? B.q[0] : B.q[1]);
  const int lane = threadIdx.x & 31;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  // the loop bound is uniform over the block, so whole warps iterate together
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nwords; base += nthr) {
    const int64_t w = base + threadIdx.x;
    uint32_t unv = 0u;
    if (w < nwords) {
      const int64_t left = (int64_t)nb - w * 32;  // vertices of this word in the graph
      const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : (left > 0 ? (1u << left) - 1u : 0u);
      unv = ~visited[w] & valid;
      fnext[w] = 0u;
    }
    const unsigned cnt = __popc(unv);
    unsigned inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, inc, 31);
    unsigned long long at = 0;
    if (lane == 31 && total) at = atomicAdd(&c->bl_len, (unsigned long long)total);
    at = __shfl_sync(0xffffffffu, at, 31);
    unsigned long long pos = at + inc - cnt;
    while (unv) {
      list[pos++] = (int32_t)(w * 32 + (__ffs(unv) - 1));
      unv &= unv - 1u;
    }
  }
}

template <int REV>
__global__ void __launch_bounds__(256) bu_list_pull(int32_t nb, int64_t nwords, uint32_t* visited,
                                                    Bufs B, const int64_t* __restrict__ off,
                                                    const int32_t* __restrict__ col,
                                                    const int2* __restrict__ nplus, PlOut plo,
                                                    Ctrl* c, int unused) {
  if (c->dir != G3_DIR_BU) return;
  const uint32_t* __restrict__ fcur = (c->fsel ? B.f[1] : B.f[0]);
  uint32_t* fnext = (c->fsel ? B.f[0] : B.f[1]);
  const int32_t* __restrict__ list = (c->qsel ? B.q[0] : B.q[1]);
  int32_t* __restrict__ fq = (c->qsel ? B.q[1] : B.q[0]);
  const int32_t lnext = c->level + 1;
  const int32_t* __restrict__ o2n = B.o2n;
  StatAcc acc;
  acc.init(c);
  const int64_t len = (int64_t)c->bl_len;
  const int lane = threadIdx.x & 31;
  // whole warps iterate together (the bound is uniform over a warp), so the
  // word grouping below may name all 32 lanes
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < len;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + lane;
    const int32_t v = i < len ? list[i] : -1;
    int32_t p = -1;
    if (v >= 0) {
      int64_t b = 0, e = 0;
      int32_t x = -1, d = 0;
      if (REV) {  // degree-aware order: the row's last entry first
        const int2 t = nplus[v];
        x = t.x;
        d = t.y;
      } else {
        b = off[v];
        e = off[v + 1];
        d = (int32_t)(e - b);
        if (d) x = col[b];
      }
      p = (x >= 0 && in_frontier(fcur, x)) ? x : -1;
      int64_t k = d > 0 ? 1 : 0;
      if (p < 0 && d > 1) {
        if (REV) {
          e = off[v + 1];
          b = e - d;
        }
        p = bu_scan_rest<REV>(col, fcur, b, e, k);
      }
      acc.ex += (unsigned)k;
      if (p >= 0) {
        pl_put(plo, v, o2n ? __ldg(&o2n[p]) : p, lnext);
        acc.add_vertex(v, d);
      }
    }
    // the list ascends within each warp's slice, so neighbouring lanes often
    // share a bitmap word: one atomic OR per distinct word and warp
    const unsigned grp = __match_any_sync(0xffffffffu, v >= 0 ? (v >> 5) : -1);
    const uint32_t bits = __reduce_or_sync(grp, p >= 0 ? 1u << (v & 31) : 0u);
    if (bits && (__ffs(grp) - 1) == lane) {
      atomicOr(&fnext[v >> 5], bits);
      atomicOr(&visited[v >> 5], bits);
    }
    const unsigned fb = __ballot_sync(0xffffffffu, p >= 0);
    if (fb) {  // one queue reservation per warp step
      unsigned long long at = 0;
      if (lane == 0) at = atomicAdd(&c->q_len, (unsigned long long)__popc(fb));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (p >= 0) fq[at + __popc(fb & g3_lanemask_lt())] = v;
    }
  }
  acc.flush(c);
}

// One round of the bottom-up search for up to U vertices per lane (v[u] < 0:
// none): first all their neighbors+ entries (last row entry and degree, 8
// coalesced bytes each; in CSR order the row bounds and first entry), then
// all their first probes, then the rest of the missed rows four entries per
// step. Found vertices get (parent, level) and their statistics; found[u]
// tells which.
template <int REV, int U>
__device__ __forceinline__ void bu_round(const int32_t (&v)[U], bool (&found)[U],
                                         const int64_t* __restrict__ off,
                                         const int32_t* __restrict__ col,
                                         const int2* __restrict__ nplus,
                                         const uint32_t* __restrict__ fcur,
                                         const int32_t* __restrict__ o2n, const PlOut& plo,
                                         int32_t lnext, StatAcc& acc) {
  int32_t x[U], d[U];
  int64_t bq[U], eq[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    x[u] = -1;
    d[u] = 0;
    bq[u] = eq[u] = 0;
  }
  if (REV) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v[u] >= 0) {
        const int2 tt = nplus[v[u]];
        x[u] = tt.x;
        d[u] = tt.y;
      }
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v[u] >= 0) {
        bq[u] = off[v[u]];
        eq[u] = off[v[u] + 1];
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      d[u] = (int32_t)(eq[u] - bq[u]);
      if (d[u] > 0) x[u] = __ldg(&col[bq[u]]);
    }
  }
  int32_t p[U];
#pragma unroll
  for (int u = 0; u < U; ++u) p[u] = (x[u] >= 0 && in_frontier(fcur, x[u])) ? x[u] : -1;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    int64_t k = d[u] > 0 ? 1 : 0;
    if (p[u] < 0 && d[u] > 1) {
      if (REV) {
        eq[u] = off[v[u] + 1];
        bq[u] = eq[u] - d[u];
      }
      p[u] = bu_scan_rest4<REV>(col, fcur, bq[u], eq[u], k);
    }
    acc.ex += (unsigned)k;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    found[u] = p[u] >= 0;
    if (found[u]) {
      pl_put(plo, v[u], o2n ? __ldg(&o2n[p[u]]) : p[u], lnext);
      acc.add_vertex(v[u], d[u]);
    }
  }
}

// Bottom-up level over word tiles (Algorithms 5 and 6). A warp owns 32
// consecutive words of the visited bitmap (1024 vertices) at a time; lane i
// reads word i, so a tile without unvisited vertices costs one coalesced
// load and one store of zero next-frontier words. A dense tile (at least
// BU_DENSE unvisited vertices) is worked lane by word: lane i takes the
// unvisited vertices of word i, U per round, and builds its next-frontier
// word in a register. A sparse tile's unvisited vertices are first compacted
// into a per-warp list in shared memory so that every lane has work; found
// vertices then set their bit in the warp's next-frontier tile in shared
// memory. Either way lane i finally writes next-frontier word i and ORs it
// into visited word i (the paper's visited |= F_next, without atomics in
// global memory).
#define BU_WARPS 8
#define BU_DENSE 384
template <int REV, int U>
__global__ void __launch_bounds__(32 * BU_WARPS, (U > 2 ? 4 : 5)) bu_tiles(
    int32_t nb, int64_t nwords, uint32_t* visited, Bufs B, const int64_t* __restrict__ off,
    const int32_t* __restrict__ col, const int2* __restrict__ nplus, PlOut plo, Ctrl* c,
    int skip_dense) {
  if (c->dir != G3_DIR_BU || (skip_dense && bu_dense(c, nb))) return;
  __shared__ uint16_t s_list[BU_WARPS][1024];
  __shared__ uint32_t s_next[BU_WARPS][32];
  const uint32_t* __restrict__ fcur = (c->fsel ? B.f[1] : B.f[0]);
  uint32_t* __restrict__ fnext = (c->fsel ? B.f[0] : B.f[1]);
  const int32_t lnext = c->level + 1;
  const int32_t* __restrict__ o2n = B.o2n;
  StatAcc acc;
  acc.init(c);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint16_t* list = s_list[wib];
  uint32_t* nx = s_next[wib];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ntiles = (nwords + 31) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += nwarps) {
    const int64_t w = t * 32 + lane;
    const int64_t vbase = t * 1024;
    uint32_t vis = 0xFFFFFFFFu, unv = 0u;
    if (w < nwords) {
      vis = visited[w];
      const int64_t left = (int64_t)nb - w * 32;  // vertices of this word in the graph
      const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
      unv = ~vis & valid;
    }
    const unsigned cnt = __popc(unv);
    const unsigned total = __reduce_add_sync(0xffffffffu, cnt);
    if (total == 0) {
      if (w < nwords) fnext[w] = 0u;
      continue;
    }
    uint32_t nword = 0u;
    if (total >= BU_DENSE) {
      // lane by word: U of this word's unvisited vertices per round
      uint32_t rem = unv;
      while (__any_sync(0xffffffffu, rem != 0u)) {
        int32_t v[U];
        int bitpos[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          bitpos[u] = rem ? __ffs(rem) - 1 : -1;
          v[u] = bitpos[u] >= 0 ? (int32_t)(w * 32 + bitpos[u]) : -1;
          if (rem) rem &= rem - 1u;
        }
        bool found[U];
        bu_round<REV, U>(v, found, off, col, nplus, fcur, o2n, plo, lnext, acc);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (found[u]) nword |= 1u << bitpos[u];
      }
    } else {
      // compact the tile's unvisited vertices (offsets within the tile)
      unsigned inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      unsigned pos = inc - cnt;
      uint32_t bits = unv;
      while (bits) {
        const int bb = __ffs(bits) - 1;
        list[pos++] = (uint16_t)(lane * 32 + bb);
        bits &= bits - 1u;
      }
      nx[lane] = 0u;
      __syncwarp();
      for (unsigned base = 0; base < total; base += 32 * U) {
        int32_t v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned j = base + u * 32 + lane;
          v[u] = j < total ? (int32_t)(vbase + list[j]) : -1;
        }
        bool found[U];
        bu_round<REV, U>(v, found, off, col, nplus, fcur, o2n, plo, lnext, acc);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (found[u]) {
            const int32_t rel = v[u] - (int32_t)vbase;
            atomicOr(&nx[rel >> 5], 1u << (rel & 31));
          }
      }
      __syncwarp();
      nword = nx[lane];
      __syncwarp();
    }
    if (w < nwords) {
      fnext[w] = nword;
      if (nword) visited[w] = vis | nword;
    }
  }
  acc.flush(c);
}

// ------------------------------------------- bottom-up, staged tiles
// Asynchronous bulk copies (the TMA unit's cp.async.bulk) into shared
// memory, completed on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for the phase with the given parity; false when it did not
// complete within `spins` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned spins) {
  for (unsigned i = 0; i < spins; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

#define BS_TILE 1024  // vertices per staged tile (32 bitmap words)
#define BS_THREADS 256
#define BS_SPINS (1u << 22)

// Test hook (g3_debug_inject, G3_INJECT_STAGED_STALL): when positive, the
// staged kernel leaves out the bulk copies of each CTA's first tile, so that
// its bounded wait on that tile's barrier runs out after this many polls.
__device__ int g3_dbg_staged_stall;

g3_status g3_bfs_set_staged_stall(int spins) {
  G3_TRY_CUDA(cudaMemcpyToSymbol(g3_dbg_staged_stall, &spins, sizeof(int)));
  return G3_OK;
}

// Dense bottom-up level with the streamed inputs staged in shared memory
// (Algorithms 5 and 6). A CTA walks tiles of 1024 vertices; while it works
// on one tile, the bulk-copy engine brings the next tile's neighbors+
// entries (8 KB) and visited words (128 B) into the other of two shared
// buffers, so the only loads left in the threads' dependent chains are the
// frontier-bitmap probes, the parents' original IDs and the rows of missed
// vertices. Warp w takes words 4w..4w+3 of the tile, one vertex per lane and
// word: the first probes of its four vertices are issued together, hits set
// their word's bits by ballot, and misses with more neighbours go to a
// per-CTA list that all threads then scan (rest of the row, four entries per
// step), so that a long row does not hold a whole warp. Each wait on a
// tile's barrier is bounded; if one runs out the CTA flags the controller
// record (the search stops with G3_ETIMEOUT), waits once more for the copy it
// issued and returns.
__global__ void __launch_bounds__(BS_THREADS, 4) bu_staged(
    int32_t nb, int64_t nwords, uint32_t* visited, Bufs B, const int64_t* __restrict__ off,
    const int32_t* __restrict__ col, const int2* __restrict__ nplus, PlOut plo, Ctrl* c) {
  if (c->dir != G3_DIR_BU || !bu_dense(c, nb)) return;
  __shared__ __align__(16) int2 s_np[2][BS_TILE];
  __shared__ __align__(16) uint32_t s_vis[2][32];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_next[32];
  __shared__ uint16_t s_pend[BS_TILE];
  __shared__ unsigned s_npend;
  const uint32_t* __restrict__ fcur = (c->fsel ? B.f[1] : B.f[0]);
  uint32_t* __restrict__ fnext = (c->fsel ? B.f[0] : B.f[1]);
  const int32_t lnext = c->level + 1;
  const int32_t* __restrict__ o2n = B.o2n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ntiles = (nwords + 31) >> 5;
  StatAcc acc;
  acc.init(c);
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // bulk copies of tile t into buffer b (sizes rounded up to 16 bytes; the
  // workspace arrays have padding past their ends)
  auto issue = [&](int64_t t, int b) {
    const int64_t v0 = t * BS_TILE, w0 = t * 32;
    const int64_t nv = min((int64_t)BS_TILE, (int64_t)nb - v0);
    const int64_t nw = min((int64_t)32, nwords - w0);
    const unsigned bnp = (unsigned)(((nv * 8) + 15) & ~15ll);
    const unsigned bvis = (unsigned)(((nw * 4) + 15) & ~15ll);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&s_bar[b], bnp + bvis);
    bulk_g2s(&s_np[b][0], nplus + v0, bnp, &s_bar[b]);
    bulk_g2s(&s_vis[b][0], visited + w0, bvis, &s_bar[b]);
  };
  const int stall = g3_dbg_staged_stall;
  const unsigned spins = stall > 0 ? (unsigned)stall : BS_SPINS;
  unsigned phases = 0u;  // bit b: parity of the next phase of buffer b
  int64_t t = blockIdx.x;
  if (tid == 0 && t < ntiles) {
    if (stall > 0) {
      mbar_expect_tx(&s_bar[0], 16);  // armed, but nothing will arrive
    } else {
      issue(t, 0);
    }
  }
  for (int k = 0; t < ntiles; ++k, t += gridDim.x) {
    const int b = k & 1;
    const int64_t tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) issue(tn, b ^ 1);
    const bool ok = mbar_wait(&s_bar[b], (phases >> b) & 1u, spins);
    phases ^= 1u << b;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&c->err, 1u);
        // the copy of the next tile is in flight: wait for it (bounded)
        if (tn < ntiles) mbar_wait(&s_bar[b ^ 1], (phases >> (b ^ 1)) & 1u, BS_SPINS);
      }
      return;
    }
    if (tid < 32) s_next[tid] = 0u;
    if (tid == 0) s_npend = 0u;
    __syncthreads();
    // first probes: warp w, words 4w .. 4w+3 of the tile, all four issued
    // before any is used
    const int64_t wbase = t * 32;
    bool cand[4], hit[4];
    int32_t x[4], d[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int wi = warp * 4 + u;
      const int64_t gw = wbase + wi;
      const int64_t v = gw * 32 + lane;
      cand[u] = gw < nwords && v < nb && !((s_vis[b][wi] >> lane) & 1u);
      x[u] = -1;
      d[u] = 0;
      if (cand[u]) {
        const int2 e = s_np[b][wi * 32 + lane];
        x[u] = e.x;
        d[u] = e.y;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) hit[u] = x[u] >= 0 && in_frontier(fcur, x[u]);
    int32_t po[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) po[u] = hit[u] ? (o2n ? __ldg(&o2n[x[u]]) : x[u]) : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int wi = warp * 4 + u;
      const int32_t v = (int32_t)((wbase + wi) * 32 + lane);
      if (cand[u] && d[u] > 0) acc.ex += 1u;
      if (hit[u]) {
        pl_put(plo, v, po[u], lnext);
        acc.add_vertex(v, d[u]);
      }
      const bool miss = cand[u] && !hit[u] && d[u] > 1;
      const unsigned mb = __ballot_sync(0xffffffffu, miss);
      unsigned base = 0;
      if (lane == 0 && mb) base = atomicAdd(&s_npend, (unsigned)__popc(mb));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (miss) s_pend[base + __popc(mb & g3_lanemask_lt())] = (uint16_t)(wi * 32 + lane);
      const unsigned hb = __ballot_sync(0xffffffffu, hit[u]);
      if (lane == 0) s_next[wi] = hb;
    }
    __syncthreads();
    // the rest of the missed rows, spread over all threads of the CTA
    const unsigned npend = s_npend;
    for (unsigned j = tid; j < npend; j += BS_THREADS) {
      const int rel = s_pend[j];
      const int64_t v = t * BS_TILE + rel;
      const int64_t e = off[v + 1];
      const int32_t d = s_np[b][rel].y;
      int64_t kk = 1;
      const int32_t p = bu_scan_rest4<1>(col, fcur, e - d, e, kk);
      acc.ex += (unsigned)(kk - 1);
      if (p >= 0) {
        pl_put(plo, (int32_t)v, o2n ? __ldg(&o2n[p]) : p, lnext);
        acc.add_vertex((int32_t)v, d);
        atomicOr(&s_next[rel >> 5], 1u << (rel & 31));
      }
    }
    __syncthreads();
    if (tid < 32) {
      const int64_t gw = wbase + tid;
      if (gw < nwords) {
        const uint32_t nw = s_next[tid];
        fnext[gw] = nw;
        if (nw) visited[gw] = s_vis[b][tid] | nw;
      }
    }
    __syncthreads();  // buffer b and the shared lists are reused
  }
  acc.flush(c);
}

// The word-tile kernel in the scan order of the options.
static void* bu_tiles_fn(int rev) {
  return rev ? (void*)bu_tiles<1, 4> : (void*)bu_tiles<0, 4>;
}

// ------------------------------------------------------------ conversions
// queue -> bitmap before a bottom-up level that follows a top-down one:
// clear f[fsel], then set the bit of every queued vertex.
__global__ void bm_clear(Bufs B, int64_t nwords, const Ctrl* c) {
  if (c->dir != G3_DIR_BU || c->fmt_queue != 1) return;
  uint32_t* f = (c->fsel ? B.f[1] : B.f[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
       i += (int64_t)gridDim.x * blockDim.x)
    f[i] = 0u;
}

__global__ void q_to_bitmap(Bufs B, const Ctrl* c) {
  if (c->dir != G3_DIR_BU || c->fmt_queue != 1) return;
  const int32_t* __restrict__ q = (c->qsel ? B.q[1] : B.q[0]);
  uint32_t* bm = (c->fsel ? B.f[1] : B.f[0]);
  const int64_t len = c->nf;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = q[i];
    atomicOr(&bm[v >> 5], 1u << (v & 31));
  }
}

// bitmap -> queue before a top-down level that follows a bottom-up one.
__global__ void bitmap_to_q(Bufs B, int64_t nwords, Ctrl* c) {
  if (c->dir != G3_DIR_TD || c->fmt_queue) return;
  const uint32_t* __restrict__ bm = (c->fsel ? B.f[1] : B.f[0]);
  int32_t* q = (c->qsel ? B.q[1] : B.q[0]);
  unsigned long long* len = &c->conv_len;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
       base < nwords; base += nwarps * 32) {
    const int64_t w = base + lane;
    uint32_t bits = w < nwords ? bm[w] : 0u;
    unsigned cnt = __popc(bits), inc = cnt;
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
    unsigned long long p = start + inc - cnt;
    while (bits) {
      int b = __ffs(bits) - 1;
      q[p++] = (int32_t)(w * 32 + b);
      bits &= bits - 1u;
    }
  }
}

// ------------------------------------------------------------- controller
// Learned controller: the 12-32-4 MLP of g3_mlp.cuh on the frontier record.
__device__ __forceinline__ int clamp_thr(float lg, int lo, int hi) {
  float x = fminf(fmaxf(rintf(lg), (float)lo), (float)hi);
  return 1 << (int)x;
}

struct CtrlArgs {
  int32_t nb;
  int64_t nnz;
  int controller, alpha, beta;
  const float* mlp;
  float mlp_margin;
  int mlp_bins;
  int t1, t2, t3;
  LevelLog* log;
  int graph_mode;
  cudaGraphConditionalHandle h_loop;
  int bu_list;  // sparse bottom-up levels run over a vertex list
  cudaGraphConditionalHandle h_mode;  // graph mode: the SWITCH of the next level
};

// After the expansion of level L: record where the produced frontier lives,
// promote it to F_{L+1}, update the visited totals, decide its direction,
// log it and clear the accumulators for the next expansion. In graph mode it
// also ends the loop (done, or the launch's level cap reached).
__global__ void bfs_control(Ctrl* c, CtrlArgs A) {
  // The record is brought into shared memory in 16-byte words, one per lane,
  // worked on there by lane 0 and written back the same way: two round trips
  // to L2 instead of one per field that lane 0 reads after writing.
  __shared__ Ctrl sc;
  __shared__ float feat[MLP_IN];
  __shared__ long long s_prev_nf;
  __shared__ int decide, active, s_dir, s_near;
  const int lane = threadIdx.x;
  MlpLane W;  // the weights are on their way while the record is updated
  if (A.controller == G3_CTRL_LEARNED) mlp_load_lane(A.mlp, W);
  constexpr int kWords = (int)(sizeof(Ctrl) / 16);
  int4* gw = reinterpret_cast<int4*>(c);
  int4* sw = reinterpret_cast<int4*>(&sc);
  for (int i = lane; i < kWords; i += 32) sw[i] = gw[i];
  __syncwarp();
  Ctrl* const r = &sc;
  if (lane == 0) {
    active = r->mode != MODE_DONE && r->nf > 0;
    if (active) {
      const int prev_dir = r->dir;
      const bool was_td = prev_dir == G3_DIR_TD;
      const long long prev_nf = r->nf;
      const long long nf = was_td ? (long long)r->q_len : (long long)r->nx_nf;
      if (was_td) {
        r->qsel ^= 1;
        r->fmt_queue = 1;
      } else {
        // a sparse level also left its next frontier in q[qsel]
        r->fsel ^= 1;
        r->fmt_queue = r->bu_sparse ? 2 : 0;
      }
      if (r->level < LOG_MAX) {
        A.log[r->level].n_next = nf;
        if (!was_td) A.log[r->level].examined = (long long)r->nx_exam;
      }
      r->nf = nf;
      r->mf = (long long)r->nx_mf;
      for (int k = 0; k < 4; ++k) r->hist[k] = (long long)r->nx_hist[k];
      r->id_min = nf ? (int)r->nx_min : 0;
      r->id_max = nf ? (int)r->nx_max : 0;
      r->n_visited += nf;
      r->m_visited += r->mf;
      r->nu = A.nb - r->n_visited;
      r->mu = A.nnz - r->m_visited;
      r->level += 1;
      int d;
      if (A.controller == G3_CTRL_TOPDOWN) {
        d = G3_DIR_TD;
      } else if (A.controller == G3_CTRL_BOTTOMUP) {
        d = G3_DIR_BU;
      } else if (prev_dir == G3_DIR_TD) {
        d = (r->mf * (long long)A.alpha > r->mu) ? G3_DIR_BU : G3_DIR_TD;
      } else {
        d = (nf < prev_nf && nf * (long long)A.beta < (long long)A.nb) ? G3_DIR_TD : G3_DIR_BU;
      }
      r->t1 = A.t1;
      r->t2 = A.t2;
      r->t3 = A.t3;
      decide = d;
      s_prev_nf = prev_nf;
      s_dir = prev_dir;
      // the network is consulted where the rule's own test is within a
      // factor of 4 of its threshold; elsewhere the rule's answer is clear
      {
        const long long lhs = was_td ? r->mf * (long long)A.alpha : nf * (long long)A.beta;
        const long long rhs = was_td ? r->mu : (long long)A.nb;
        s_near = 4 * lhs > rhs && lhs < 4 * rhs;
      }
      for (int k = 0; k < 4; ++k) r->mlp_out[k] = 0.f;  // (the network's, if consulted)
      reset_next(r);
    }
  }
  __syncwarp();
  if (active && A.controller == G3_CTRL_LEARNED && s_near) {
    // lane j computes feature j, all twelve at once
    if (lane < MLP_IN)
      feat[lane] = mlp_feature(lane, r->nf, r->mf, r->nu, r->mu, A.nb, A.nnz, s_dir, r->level,
                               s_prev_nf);
    __syncwarp();
    float out[4];
    mlp_eval_lane(W, feat, out);
    if (lane == 0) {
      for (int k = 0; k < 4; ++k) r->mlp_out[k] = out[k];
      // inside the margin the alpha/beta rule's direction stands
      if (fabsf(out[0]) > A.mlp_margin) decide = out[0] < 0.f ? G3_DIR_BU : G3_DIR_TD;
      if (A.mlp_bins) {
        int a1 = clamp_thr(out[1], 2, 12), a2 = clamp_thr(out[2], 6, 18),
            a3 = clamp_thr(out[3], 10, 26);
        if (a2 <= a1) a2 = a1 * 2;
        if (a3 <= a2) a3 = a2 * 2;
        r->t1 = a1;
        r->t2 = a2;
        r->t3 = a3;
      }
    }
    __syncwarp();
  }
  if (lane == 0 && active) {
    r->dir = decide;
    r->bu_sparse = decide == G3_DIR_BU && A.bu_list && bu_sparse_level(r->nu, A.nb);
    r->mode = r->err ? MODE_DONE : mode_of(r);
    if (r->mode != MODE_DONE) log_frontier(A.log, r);
  }
  __syncwarp();
  for (int i = lane; i < kWords; i += 32) gw[i] = sw[i];
  if (lane == 0 && A.graph_mode) {
    // the level just decided runs in this loop iteration, unless the search
    // is done or has reached the launch's level cap (the host then goes on
    // from this record)
    const bool go = r->mode != MODE_DONE && r->level < r->cap;
    cudaGraphSetConditional(A.h_mode, go ? (unsigned)r->mode : (unsigned)MODE_DONE);
    cudaGraphSetConditional(A.h_loop, go ? 1u : 0u);
  }
}



// --------------------------------------------------------- output mapping
// Whether label x was reached. A search reaches exactly its root's connected
// component, and after a full RCM relabel that component is one range of
// labels, so the test is two compares instead of a probe of the visited
// bitmap (a random 4-byte read per vertex, half of this pass's L2 requests).
struct Reach {
  const uint32_t* visited;
  int32_t nb, lo, hi;
  int ok;
};

__device__ __forceinline__ Reach reach_of(const Ctrl* c, const uint32_t* visited, int32_t nb) {
  return Reach{visited, nb, c->rng_lo, c->rng_hi, c->rng_ok};
}

__device__ __forceinline__ bool reached(const Reach& R, int32_t x) {
  if (R.ok) return x >= R.lo && x < R.hi;
  return x < R.nb && ((__ldg(&R.visited[x >> 5]) >> (x & 31)) & 1u);
}

__global__ void bfs_translate(int32_t n, int32_t nb, int32_t root,
                              const int32_t* __restrict__ new_of_old,
                              const uint32_t* __restrict__ visited, const Ctrl* c, PlOut plo,
                              int32_t* parent, int32_t* level) {
  const Reach R = reach_of(c, visited, nb);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = -1, l = -1;
    const int32_t x = new_of_old ? new_of_old[v] : (int32_t)v;
    if (reached(R, x)) {
      const int2 t = pl_decode(plo, plo.pl[x], x);
      p = t.x;
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

// Same mapping, four consecutive original IDs per thread: one 128-bit load
// of new_of_old, four independent gathers of the packed (parent, level) word
// in flight at once (the random gathers are what bounds this pass, so their
// latency has to overlap), 128-bit stores. The streamed input and the outputs
// carry evict-first hints so that L2 keeps the gathered words. parent and
// level must be 16-byte aligned.
__global__ void __launch_bounds__(256) bfs_translate4(int32_t n, int32_t nb, int32_t root,
                                                      const int32_t* __restrict__ new_of_old,
                                                      const uint32_t* __restrict__ visited,
                                                      const Ctrl* c, PlOut plo, int32_t* parent,
                                                      int32_t* level) {
  const Reach R = reach_of(c, visited, nb);
  const int64_t n4 = n >> 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x[4];
    if (new_of_old) {
      // streamed once: evict-first, so the packed words stay in L2
      const int4 xs = __ldcs(reinterpret_cast<const int4*>(new_of_old) + i);
      x[0] = xs.x;
      x[1] = xs.y;
      x[2] = xs.z;
      x[3] = xs.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = (int)(4 * i + k);
    }
    bool r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = reached(R, x[k]);
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = r[k] ? __ldg(&plo.pl[x[k]]) : 0u;
    int p[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int2 t = r[k] ? pl_decode(plo, w[k], x[k]) : make_int2(-1, -1);
      p[k] = t.x;
      l[k] = t.y;
    }
    if ((root >> 2) == i) {
      p[root & 3] = root;
      l[root & 3] = 0;
    }
    __stcs(reinterpret_cast<int4*>(parent) + i, make_int4(p[0], p[1], p[2], p[3]));
    __stcs(reinterpret_cast<int4*>(level) + i, make_int4(l[0], l[1], l[2], l[3]));
  }
  // the last n % 4 IDs
  const int64_t v = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < n) {
    int32_t p = -1, l = -1;
    const int32_t xv = new_of_old ? new_of_old[v] : (int32_t)v;
    if (reached(R, xv)) {
      const int2 t = pl_decode(plo, plo.pl[xv], xv);
      p = t.x;
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

// The same mapping in two passes over label halves, for packed arrays too
// large to stay in L2 beside the streamed arrays (at 2^26 vertices the
// packed words take 131 MB, and one pass gathering from all of them misses
// L2 on most 4-byte gathers, each costing a 32-byte sector). Pass 1 streams
// new_of_old and resolves the vertices labelled below `split`, gathering only
// from that half of the packed array; for every original ID it writes one
// 4-byte record into parent[] (used as scratch): the packed word itself
// (parent, level code) when resolved, or a marker. Pass 2 streams those
// records, resolves the rest from the other half, and writes parent[] and
// level[]. Records use the packed format with three reserved level codes
// (lmax = 2^bits - 1): lmax - 1 unreached or isolated, lmax pending with the
// label in the parent field; resolved levels are below lmax - 1 (higher
// levels, and those in the side table, are left pending for pass 2, which
// decodes them from the packed word). Needs bits >= 4 and 16-byte aligned
// outputs.
__device__ __forceinline__ uint32_t tr_pass1_one(int32_t x, int32_t split, const Reach& R,
                                                 const PlOut& plo, uint32_t lmax) {
  if (!reached(R, x)) return lmax - 1u;
  const uint32_t pend = ((uint32_t)x << plo.bits) | lmax;
  if (x >= split) return pend;
  const uint32_t w = __ldg(&plo.pl[x]);
  return (w & lmax) < lmax - 1u ? w : pend;
}

__global__ void __launch_bounds__(256) bfs_translate_p1(int32_t n, int32_t nb, int32_t split,
                                                        const int32_t* __restrict__ new_of_old,
                                                        const uint32_t* __restrict__ visited,
                                                        const Ctrl* c, PlOut plo,
                                                        uint32_t* rec) {
  const Reach R = reach_of(c, visited, nb);
  const uint32_t lmax = (1u << plo.bits) - 1u;
  const int64_t n4 = n >> 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 xs = __ldcs(reinterpret_cast<const int4*>(new_of_old) + i);
    uint4 r;
    r.x = tr_pass1_one(xs.x, split, R, plo, lmax);
    r.y = tr_pass1_one(xs.y, split, R, plo, lmax);
    r.z = tr_pass1_one(xs.z, split, R, plo, lmax);
    r.w = tr_pass1_one(xs.w, split, R, plo, lmax);
    __stcs(reinterpret_cast<uint4*>(rec) + i, r);
  }
  const int64_t v = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < n) rec[v] = tr_pass1_one(new_of_old[v], split, R, plo, lmax);
}

__device__ __forceinline__ int2 tr_pass2_one(uint32_t r, const PlOut& plo, uint32_t lmax) {
  const uint32_t code = r & lmax;
  if (code == lmax - 1u) return make_int2(-1, -1);
  if (code == lmax) {
    const int32_t x = (int32_t)(r >> plo.bits);
    return pl_decode(plo, __ldg(&plo.pl[x]), x);
  }
  return make_int2((int32_t)(r >> plo.bits), (int32_t)code);
}

__global__ void __launch_bounds__(256) bfs_translate_p2(int32_t n, int32_t root, PlOut plo,
                                                        int32_t* parent, int32_t* level) {
  const uint32_t lmax = (1u << plo.bits) - 1u;
  const int64_t n4 = n >> 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = __ldcs(reinterpret_cast<const uint4*>(parent) + i);
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    // the pending ones first, so that their gathers are in flight together
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[k] = (rr[k] & lmax) == lmax ? __ldg(&plo.pl[rr[k] >> plo.bits]) : 0u;
    int p[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t code = rr[k] & lmax;
      int2 t;
      if (code == lmax) t = pl_decode(plo, w[k], (int32_t)(rr[k] >> plo.bits));
      else if (code == lmax - 1u) t = make_int2(-1, -1);
      else t = make_int2((int32_t)(rr[k] >> plo.bits), (int32_t)code);
      p[k] = t.x;
      l[k] = t.y;
    }
    if ((root >> 2) == i) {
      p[root & 3] = root;
      l[root & 3] = 0;
    }
    __stcs(reinterpret_cast<int4*>(parent) + i, make_int4(p[0], p[1], p[2], p[3]));
    __stcs(reinterpret_cast<int4*>(level) + i, make_int4(l[0], l[1], l[2], l[3]));
  }
  const int64_t v = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < n) {
    int2 t = tr_pass2_one((uint32_t)parent[v], plo, lmax);
    if (v == root) t = make_int2(root, 0);
    parent[v] = t.x;
    level[v] = t.y;
  }
}

__global__ void build_nplus(int32_t nb, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ col, int2* nplus) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nb;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[v], e = off[v + 1];
    nplus[v] = make_int2(e > b ? col[e - 1] : -1, (int32_t)(e - b));
  }
}

// ------------------------------------------------------------------ host
extern "C" void g3_bfs_opts_default(g3_bfs_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->controller = G3_CTRL_HEURISTIC;
  o->mlp_bins = 1;
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
  ws->plo.bits = pl_bits(g->n);
  ws->nwords = ((int64_t)g->n_bfs + 31) / 32;
  const size_t nb1 = (size_t)g->n_bfs + 4, nw = (size_t)ws->nwords + 4, n1 = (size_t)g->n + 4;
  struct {
    void** p;
    size_t bytes;
  } req[] = {
      {(void**)&ws->visited, nw * 4},        {(void**)&ws->fa, nw * 4},
      {(void**)&ws->fb, nw * 4},             {(void**)&ws->vis_save, nw * 4},
      {(void**)&ws->qa, nb1 * 4},            {(void**)&ws->qb, nb1 * 4},
      {(void**)&ws->bins, nb1 * 4 * 3},      {(void**)&ws->plo.pl, nb1 * 4},
      {(void**)&ws->plo.deep, nb1 * 4},
      {(void**)&ws->nplus, nb1 * 8},
      {(void**)&ws->goff, nb1 * 8},          {(void**)&ws->out_parent, n1 * 4},
      {(void**)&ws->out_level, n1 * 4},
      {(void**)&ws->ctrl, sizeof(Ctrl)},
      {(void**)&ws->log, sizeof(LevelLog) * LOG_MAX},
  };
  for (auto& r : req) {
    cudaError_t e = g3_alloc_should_fail() ? cudaErrorMemoryAllocation
                                            : cudaMalloc(r.p, r.bytes);
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
  if (ws->nb > 0) {  // neighbors+ (Algorithm 6): last row entry and degree
    build_nplus<<<g3_grid_for(ws->nb, 256), 256>>>(ws->nb, g->off, g->col, ws->nplus);
    g3_count_launch();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      g3_set_error("g3_bfs workspace: %s", cudaGetErrorString(e));
      g3_bfs_ws_free(ws);
      return G3_ECUDA;
    }
  }
  ws->grid_front = resident_grid(td_front, 256);
  ws->grid_bins = resident_grid(td_bins, 256);
  ws->grid_bu = resident_grid(bu_pull<1, 0>, 256);
  int g0 = resident_grid(bu_pull<0, 0>, 256);
  if (g0 < ws->grid_bu) ws->grid_bu = g0;
  g0 = resident_grid(bu_pull<1, 1>, 256);
  if (g0 < ws->grid_bu) ws->grid_bu = g0;
  g0 = resident_grid(bu_pull<0, 1>, 256);
  if (g0 < ws->grid_bu) ws->grid_bu = g0;
  ws->grid_tiles = resident_grid(bu_tiles<1, 4>, 32 * BU_WARPS);
  g0 = resident_grid(bu_tiles<0, 4>, 32 * BU_WARPS);
  if (g0 < ws->grid_tiles) ws->grid_tiles = g0;
  ws->grid_staged = resident_grid(bu_staged, BS_THREADS);
  ws->grid_conv = resident_grid(bitmap_to_q, 256);
  ws->grid_lb = resident_grid(bu_list_build, 256);
  ws->grid_lp = resident_grid(bu_list_pull<1>, 256);
  g0 = resident_grid(bu_list_pull<0>, 256);
  if (g0 < ws->grid_lp) ws->grid_lp = g0;
  ws->grid_tr = resident_grid(bfs_translate, 256);
  ws->grid_tr4 = resident_grid(bfs_translate4, 256);
  *out = ws;
  return G3_OK;
}

// A pointer the device can write for p: p itself for device or managed
// memory, the device alias of page-locked host memory (the output pass then
// writes straight into host memory over the chip-to-chip link), NULL for
// pageable host memory (which goes through a device staging buffer).
static int32_t* device_view(int32_t* p, bool* in_hbm = nullptr) {
  cudaPointerAttributes at;
  if (in_hbm) *in_hbm = false;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice) {
    if (in_hbm) *in_hbm = true;
    return p;
  }
  if (at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) return (int32_t*)at.devicePointer;
  return nullptr;
}


static inline int cap_grid(int64_t items, int per_block, int resident) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b > resident) b = resident;
  return b < 1 ? 1 : (int)b;
}

// Everything the expansion kernels of one search take as arguments.
struct Launch {
  g3_graph* g;
  g3_bfs_ws* ws;
  const g3_bfs_opts* o;
  Bufs B;
  int64_t nb1;
  int full_stats;  // the kernels keep the per-level histogram and label range
};

// The word-pair bottom-up kernel for a scan order and statistics mode.
static void* bu_pull_fn(int rev, int full) {
  return rev ? (full ? (void*)bu_pull<1, 1> : (void*)bu_pull<1, 0>)
             : (full ? (void*)bu_pull<0, 1> : (void*)bu_pull<0, 0>);
}

static bool bu_uses_list(const g3_bfs_opts& o) { return o.bu_kernel == 0; }

static CtrlArgs ctrl_args(const Launch& S, int graph_mode, cudaGraphConditionalHandle h_loop,
                          cudaGraphConditionalHandle h_mode) {
  return CtrlArgs{S.ws->nb,     S.g->nnz,        S.o->controller,
                  S.o->alpha,   S.o->beta,       S.o->mlp_params,
                  S.o->mlp_margin * 1e-3f,       S.o->mlp_bins,   S.o->t1,
                  S.o->t2,      S.o->t3,         S.ws->log,
                  graph_mode,   h_loop,          bu_uses_list(*S.o), h_mode};
}

// Which bottom-up kernels the options select: bu_kernel 0 (default) word
// pairs on dense levels and the vertex-list kernels on sparse ones; 1 the
// staged kernel on dense levels and the
// word-tile kernel on the others when rows are scanned in the degree-aware
// order (word pairs in CSR order); 2 word tiles on every level; 3 word pairs
// on dense levels and word tiles on the others. Where two kernels share a
// level kind, each returns at once on the levels that are the other's.
static bool bu_uses_staged(const g3_bfs_opts& o) { return o.bu_kernel == 1 && o.bu_reverse; }
static bool bu_uses_tiles(const g3_bfs_opts& o) {
  return o.bu_kernel == 2 || o.bu_kernel == 3 || bu_uses_staged(o);
}
static bool bu_uses_pairs(const g3_bfs_opts& o) {
  return o.bu_kernel == 3 || !bu_uses_tiles(o);
}
// the flag both kernels of a split level kind get (skip_dense, sparse_to_tiles)
static int bu_split(const g3_bfs_opts& o) { return bu_uses_staged(o) || o.bu_kernel == 3; }
static int bu_tiles_grid(const g3_bfs_ws* ws) {
  return cap_grid((ws->nwords + 31) / 32, BU_WARPS, ws->grid_tiles);
}
static int bu_staged_grid(const g3_bfs_ws* ws) {
  return cap_grid((ws->nwords + 31) / 32, 1, ws->grid_staged);
}

// Host-driven launch of the kernels of one level of the given mode. Every
// kernel checks the controller record itself, so the set is the same as in
// the graph's SWITCH body for that mode. Records ev_mid after the format
// conversion when given.
static g3_status launch_level(const Launch& S, int mode, int64_t nf, cudaEvent_t ev_mid,
                              cudaStream_t s) {
  g3_bfs_ws* ws = S.ws;
  Ctrl* c = ws->ctrl;
  if (mode == MODE_TD_B) {
    bitmap_to_q<<<cap_grid(ws->nwords, 256, ws->grid_conv), 256, 0, s>>>(S.B, ws->nwords, c);
    G3_CHECK_LAUNCH();
  } else if (mode == MODE_BU_Q || mode == MODE_BU_QS) {
    bm_clear<<<g3_grid_for(ws->nwords, 256), 256, 0, s>>>(S.B, ws->nwords, c);
    G3_CHECK_LAUNCH();
    q_to_bitmap<<<g3_grid_for(nf, 256), 256, 0, s>>>(S.B, c);
    G3_CHECK_LAUNCH();
  }
  if (ev_mid) G3_TRY_CUDA(cudaEventRecord(ev_mid, s));
  if (mode == MODE_TD_Q || mode == MODE_TD_B || mode == MODE_TD_QS) {
    const bool small = mode == MODE_TD_QS;
    td_front<<<small ? TD_SMALL_GRID : cap_grid(nf, 256, ws->grid_front), 256, 0, s>>>(
        S.g->off, S.g->col, ws->visited, ws->plo, S.B, ws->bins, ws->goff, S.nb1, c);
    G3_CHECK_LAUNCH();
    td_bins<<<small ? TD_SMALL_GRID : ws->grid_bins, 256, 0, s>>>(
        S.g->off, S.g->col, ws->visited, ws->plo, S.B, ws->bins, ws->goff, S.nb1, c);
    G3_CHECK_LAUNCH();
  } else if (mode == MODE_BU_BS || mode == MODE_BU_QS) {
    bu_list_build<<<cap_grid(ws->nwords, 256, ws->grid_lb), 256, 0, s>>>(S.B, ws->nwords, ws->nb,
                                                                         ws->visited, c);
    G3_CHECK_LAUNCH();
    if (S.o->bu_reverse)
      bu_list_pull<1><<<ws->grid_lp, 256, 0, s>>>(ws->nb, ws->nwords, ws->visited, S.B, S.g->off,
                                                  S.g->col, ws->nplus, ws->plo, c, 0);
    else
      bu_list_pull<0><<<ws->grid_lp, 256, 0, s>>>(ws->nb, ws->nwords, ws->visited, S.B, S.g->off,
                                                  S.g->col, ws->nplus, ws->plo, c, 0);
    G3_CHECK_LAUNCH();
  } else {
    int64_t nwords = ws->nwords;
    int32_t nb = ws->nb;
    const int64_t* off = S.g->off;
    const int32_t* col = S.g->col;
    Bufs B = S.B;
    int split = bu_split(*S.o);
    void* args[] = {&nb, &nwords, &ws->visited, &B, &off, &col, &ws->nplus, &ws->plo, &c, &split};
    if (bu_uses_staged(*S.o)) {
      G3_TRY_CUDA(cudaLaunchKernel((void*)bu_staged, dim3(bu_staged_grid(ws)), dim3(BS_THREADS),
                                   args, 0, s));
      g3_count_launch();
    }
    if (bu_uses_pairs(*S.o)) {
      void* fn = bu_pull_fn(S.o->bu_reverse, S.full_stats);
      G3_TRY_CUDA(cudaLaunchKernel(fn, dim3(cap_grid(ws->nwords, 16, ws->grid_bu)), dim3(256),
                                   args, 0, s));
      g3_count_launch();
    }
    if (bu_uses_tiles(*S.o)) {
      G3_TRY_CUDA(cudaLaunchKernel(bu_tiles_fn(S.o->bu_reverse), dim3(bu_tiles_grid(ws)),
                                   dim3(32 * BU_WARPS), args, 0, s));
      g3_count_launch();
    }
  }
  return G3_OK;
}

// ------------------------------------------------------------ graph mode
static g3_status add_kernel(cudaGraph_t gr, cudaGraphNode_t* node, cudaGraphNode_t* dep,
                            void* func, int grid, int block, void** args) {
  cudaKernelNodeParams p;
  memset(&p, 0, sizeof(p));
  p.func = func;
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.kernelParams = args;
  G3_TRY_CUDA(cudaGraphAddKernelNode(node, gr, dep, dep ? 1 : 0, &p));
  return G3_OK;
}

// Zero-filled storage for cudaGraphNodeParams (its union has no usable
// default constructor).
struct NodeParams {
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  NodeParams() { memset(raw, 0, sizeof(raw)); }
  cudaGraphNodeParams& get() { return *reinterpret_cast<cudaGraphNodeParams*>(raw); }
};

static bool same_opts(const g3_bfs_opts& a, const g3_bfs_opts& b) {
  return a.controller == b.controller && a.alpha == b.alpha && a.beta == b.beta &&
         a.t1 == b.t1 && a.t2 == b.t2 && a.t3 == b.t3 && a.bu_reverse == b.bu_reverse &&
         a.mlp_params == b.mlp_params && a.mlp_margin == b.mlp_margin &&
         a.mlp_bins == b.mlp_bins && a.bu_kernel == b.bu_kernel;
}

// Builds the level loop: level 0's top-down kernels, then WHILE(h_loop) {
// bfs_control -> SWITCH(h_mode) { TD_Q, TD_B, BU_B, BU_Q, -, BU_BS, BU_QS } }:
// the controller closes the level just expanded and sets both conditions for
// the next one. Kernel arguments are baked in; everything that changes per
// search lives in the controller record.
static g3_status build_graph(Launch& S) {
  g3_bfs_ws* ws = S.ws;
  cudaGraph_t top = nullptr;
  g3_status st = G3_OK;
  G3_TRY_CUDA(cudaGraphCreate(&top, 0));
  cudaGraphConditionalHandle h_loop, h_mode;
  cudaGraphNode_t wnode, sw, ctl, n0, n1, n2;
  cudaGraph_t body, br[MODE_COUNT];
  Ctrl* c = ws->ctrl;
  int64_t nwords = ws->nwords;
  int32_t nb = ws->nb;
  int gconv = ws->grid_conv, gfront = ws->grid_front, gbins = ws->grid_bins;
  const bool tiles = bu_uses_tiles(*S.o), staged = bu_uses_staged(*S.o);
  const bool pairs = bu_uses_pairs(*S.o);
  const int gtl = bu_tiles_grid(ws), gpr = cap_grid(ws->nwords, 16, ws->grid_bu);
  const int gst = bu_staged_grid(ws);
  int skip = bu_split(*S.o);
  int gclear = g3_grid_for(ws->nwords, 256), gq2b = g3_grid_for(ws->nb, 256);
  const int64_t* off = S.g->off;
  const int32_t* col = S.g->col;
  void* tiles_fn = bu_tiles_fn(S.o->bu_reverse);
  void* lp_fn = S.o->bu_reverse ? (void*)bu_list_pull<1> : (void*)bu_list_pull<0>;
  const int glb = cap_grid(ws->nwords, 256, ws->grid_lb);
  void* pairs_fn = bu_pull_fn(S.o->bu_reverse, S.full_stats);
  void* a_conv[] = {&S.B, &nwords, &c};
  void* a_clear[] = {&S.B, &nwords, &c};
  void* a_q2b[] = {&S.B, &c};
  void* a_lb[] = {&S.B, &nwords, &nb, &ws->visited, &c};
  void* a_td[] = {&off, &col, &ws->visited, &ws->plo, &S.B, &ws->bins, &ws->goff, &S.nb1, &c};
  void* a_bu[] = {&nb, &nwords, &ws->visited, &S.B, &off, &col, &ws->nplus, &ws->plo, &c,
                  &skip};
  CtrlArgs ca;
  void* a_ctl[] = {&c, &ca};
  do {
    // level 0 (top-down from the root, set up by bfs_root) runs before the
    // loop; each loop iteration then runs the controller on the level just
    // expanded, which picks the next level's SWITCH branch and whether the
    // loop goes on, and that level's kernels
    cudaGraphNode_t l0a, l0b;
    if ((st = add_kernel(top, &l0a, nullptr, (void*)td_front, gfront, 256, a_td))) break;
    if ((st = add_kernel(top, &l0b, &l0a, (void*)td_bins, gbins, 256, a_td))) break;
    if (cudaGraphConditionalHandleCreate(&h_loop, top, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess) { st = G3_ECUDA; break; }
    NodeParams wbuf;
    cudaGraphNodeParams& wp = wbuf.get();
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    if (cudaGraphAddNode(&wnode, top, &l0b, nullptr, 1, &wp) != cudaSuccess) {
      st = G3_ECUDA;
      break;
    }
    body = wp.conditional.phGraph_out[0];
    // set by the controller before every SWITCH it precedes
    if (cudaGraphConditionalHandleCreate(&h_mode, body, MODE_DONE, 0) != cudaSuccess) {
      st = G3_ECUDA;
      break;
    }
    ca = ctrl_args(S, 1, h_loop, h_mode);
    if ((st = add_kernel(body, &ctl, nullptr, (void*)bfs_control, 1, 32, a_ctl))) break;
    NodeParams sbuf;
    cudaGraphNodeParams& sp = sbuf.get();
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = h_mode;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = MODE_COUNT;  // branch MODE_DONE stays empty
    if (cudaGraphAddNode(&sw, body, &ctl, nullptr, 1, &sp) != cudaSuccess) {
      st = G3_ECUDA;
      break;
    }
    for (int k = 0; k < MODE_COUNT; ++k) br[k] = sp.conditional.phGraph_out[k];
    // MODE_TD_Q, and MODE_TD_QS on a small grid
    if ((st = add_kernel(br[MODE_TD_Q], &n0, nullptr, (void*)td_front, gfront, 256, a_td))) break;
    if ((st = add_kernel(br[MODE_TD_Q], &n1, &n0, (void*)td_bins, gbins, 256, a_td))) break;
    if ((st = add_kernel(br[MODE_TD_QS], &n0, nullptr, (void*)td_front, TD_SMALL_GRID, 256,
                         a_td)))
      break;
    if ((st = add_kernel(br[MODE_TD_QS], &n1, &n0, (void*)td_bins, TD_SMALL_GRID, 256, a_td)))
      break;
    // MODE_TD_B
    if ((st = add_kernel(br[MODE_TD_B], &n0, nullptr, (void*)bitmap_to_q, gconv, 256, a_conv)))
      break;
    if ((st = add_kernel(br[MODE_TD_B], &n1, &n0, (void*)td_front, gfront, 256, a_td))) break;
    if ((st = add_kernel(br[MODE_TD_B], &n2, &n1, (void*)td_bins, gbins, 256, a_td))) break;
    // MODE_BU_B and MODE_BU_Q (the latter after the queue -> bitmap
    // conversion): the bottom-up kernels in a chain
    if ((st = add_kernel(br[MODE_BU_Q], &n0, nullptr, (void*)bm_clear, gclear, 256, a_clear)))
      break;
    if ((st = add_kernel(br[MODE_BU_Q], &n1, &n0, (void*)q_to_bitmap, gq2b, 256, a_q2b))) break;
    for (int q = 0; q < 2 && st == G3_OK; ++q) {
      cudaGraph_t b = br[q ? MODE_BU_Q : MODE_BU_B];
      cudaGraphNode_t prev = n1, cur;
      cudaGraphNode_t* dep = q ? &prev : nullptr;
      if (staged) {
        if ((st = add_kernel(b, &cur, dep, (void*)bu_staged, gst, BS_THREADS, a_bu))) break;
        prev = cur;
        dep = &prev;
      }
      if (pairs) {
        if ((st = add_kernel(b, &cur, dep, pairs_fn, gpr, 256, a_bu))) break;
        prev = cur;
        dep = &prev;
      }
      if (tiles) {
        if ((st = add_kernel(b, &cur, dep, tiles_fn, gtl, 32 * BU_WARPS, a_bu))) break;
      }
    }
    if (st != G3_OK) break;
    // MODE_BU_BS and MODE_BU_QS (sparse levels): list, then one thread per
    // listed vertex
    if ((st = add_kernel(br[MODE_BU_QS], &n0, nullptr, (void*)bm_clear, gclear, 256, a_clear)))
      break;
    if ((st = add_kernel(br[MODE_BU_QS], &n1, &n0, (void*)q_to_bitmap, gq2b, 256, a_q2b))) break;
    if ((st = add_kernel(br[MODE_BU_QS], &n2, &n1, (void*)bu_list_build, glb, 256, a_lb))) break;
    if ((st = add_kernel(br[MODE_BU_QS], &n0, &n2, lp_fn, ws->grid_lp, 256, a_bu))) break;
    if ((st = add_kernel(br[MODE_BU_BS], &n0, nullptr, (void*)bu_list_build, glb, 256, a_lb)))
      break;
    if ((st = add_kernel(br[MODE_BU_BS], &n1, &n0, lp_fn, ws->grid_lp, 256, a_bu))) break;
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, top, 0) != cudaSuccess) {
      st = G3_ECUDA;
      break;
    }
    if (ws->gexec) cudaGraphExecDestroy(ws->gexec);
    ws->gexec = ex;
    ws->gopts = *S.o;
    ws->gfull = S.full_stats;
  } while (0);
  if (st != G3_OK) {
    cudaError_t e = cudaGetLastError();
    g3_set_error("g3_bfs: building the level-loop graph failed: %s", cudaGetErrorString(e));
  }
  cudaGraphDestroy(top);
  return st;
}

// Candidate top-down bin thresholds timed in record_both mode.
static const int kSweep[5][3] = {
    {8, 256, 8192}, {16, 512, 16384}, {32, 1024, 32768}, {64, 2048, 65536}, {128, 4096, 131072}};

// record_both mode: time every candidate top-down expansion and the
// bottom-up one from the same state, restoring the visited bitmap and the
// controller record after each trial. Fills r (times, best thresholds); the
// state afterwards is the state before the trials.
static g3_status record_trials(const Launch& S, int64_t nf, g3_level_stats* r, cudaStream_t s) {
  g3_bfs_ws* ws = S.ws;
  const size_t vbytes = (size_t)ws->nwords * 4;
  G3_TRY_CUDA(cudaMemcpyAsync(ws->vis_save, ws->visited, vbytes, cudaMemcpyDeviceToDevice, s));
  Ctrl save;
  G3_TRY_CUDA(cudaMemcpyAsync(&save, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  // a sparse bottom-up trial writes its found vertices over q[qsel], which
  // may hold the current frontier: it is kept in the output staging buffer
  // (unused until the output pass) and put back after that trial
  int32_t* qcur = S.B.q[save.qsel];
  const size_t qbytes = save.fmt_queue && nf > 0 ? (size_t)nf * 4 : 0;
  if (qbytes)
    G3_TRY_CUDA(cudaMemcpyAsync(ws->out_level, qcur, qbytes, cudaMemcpyDeviceToDevice, s));
  float best = 1e30f;
  for (int k = 0; k < 6; ++k) {
    Ctrl c = save;
    const bool td = k < 5;
    c.dir = td ? G3_DIR_TD : G3_DIR_BU;
    if (td) {
      c.t1 = kSweep[k][0];
      c.t2 = kSweep[k][1];
      c.t3 = kSweep[k][2];
    }
    c.bu_sparse = !td && bu_uses_list(*S.o) && bu_sparse_level(c.nu, ws->nb);
    const bool only_queue = c.fmt_queue == 1;
    const bool small = c.nf <= TD_SMALL_NF && c.mf <= TD_SMALL_MF;
    const int mode = td ? (c.fmt_queue ? (small ? MODE_TD_QS : MODE_TD_Q) : MODE_TD_B)
                        : c.bu_sparse ? (only_queue ? MODE_BU_QS : MODE_BU_BS)
                                      : (only_queue ? MODE_BU_Q : MODE_BU_B);
    G3_TRY_CUDA(cudaMemcpyAsync(ws->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    G3_TRY_CUDA(cudaEventRecord(ws->ev[4], s));
    G3_TRY(launch_level(S, mode, nf, nullptr, s));
    G3_TRY_CUDA(cudaEventRecord(ws->ev[5], s));
    G3_TRY_CUDA(cudaMemcpyAsync(ws->visited, ws->vis_save, vbytes, cudaMemcpyDeviceToDevice, s));
    if (!td && qbytes)
      G3_TRY_CUDA(cudaMemcpyAsync(qcur, ws->out_level, qbytes, cudaMemcpyDeviceToDevice, s));
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

static void fill_record(g3_level_stats* r, int32_t L, const LevelLog& e) {
  r->level = L;
  r->dir = e.dir;
  r->n_f = e.nf;
  r->m_f = e.mf;
  r->n_u = e.nu;
  r->m_u = e.mu;
  r->examined = e.examined;
  r->n_next = e.n_next;
  r->id_min = e.id_min;
  r->id_max = e.id_max;
  for (int k = 0; k < 4; ++k) {
    r->hist[k] = e.hist[k];
    r->mlp_out[k] = e.mlp_out[k];
  }
  r->t1 = e.t1;
  r->t2 = e.t2;
  r->t3 = e.t3;
}

// Several roots (device array) instead of one: see bfs_roots_multi.
struct MultiRoots {
  const int32_t* roots;
  int32_t count;
  const int32_t* lo;
};

static g3_status bfs_impl(g3_graph* g, int32_t root, const g3_bfs_opts* o, int32_t* parent,
                          int32_t* level, g3_level_stats* stats, int32_t max_stats,
                          int32_t* n_levels, cudaStream_t s, const MultiRoots* mr = nullptr) {
  if (!g->ws) G3_TRY(ws_create(g, &g->ws));
  g3_bfs_ws* ws = g->ws;
  const int32_t nb = ws->nb;
  Ctrl* h = ws->h_ctrl;
  const int full_stats = o->record_both || (stats && max_stats > 0 && !o->stats_counts_only);
  Launch S{g, ws, o,
           Bufs{{ws->qa, ws->qb}, {ws->fa, ws->fb}, g->relabelled ? g->old_of_new : nullptr},
           (int64_t)ws->nb + 4, full_stats};
  const bool host_driven = o->timing || o->record_both;
  if (stats && max_stats > 0) memset(stats, 0, sizeof(g3_level_stats) * (size_t)max_stats);

  G3_TRY_CUDA(cudaMemsetAsync(ws->visited, 0, (size_t)(ws->nwords + 1) * 4, s));
  const int cap = host_driven ? 0x7fffffff : GRAPH_LEVEL_CAP;
  if (mr) {
    bfs_roots_multi<<<1, 1024, 0, s>>>(mr->roots, mr->count, mr->lo,
                                       g->relabelled ? g->new_of_old : nullptr, nb, g->nnz,
                                       g->off, ws->visited, ws->plo, ws->qa, ws->ctrl, ws->log,
                                       o->t1, o->t2, o->t3, cap, full_stats);
    root = -1;  // the output pass has no single root to patch
  } else {
    bfs_root<<<1, 1, 0, s>>>(g->relabelled ? g->new_of_old : nullptr, g->comp_rng, root, nb,
                             g->nnz, g->off,
                             ws->visited, ws->plo, ws->qa, ws->ctrl, ws->log, o->t1, o->t2,
                             o->t3, cap, full_stats);
  }
  G3_CHECK_LAUNCH();

  // outputs in original IDs: device (or device-visible host) buffers, else
  // staging buffers copied to the host at the end
  bool hbm_p = false, hbm_l = false;
  int32_t* vp = device_view(parent, &hbm_p);
  int32_t* vl = device_view(level, &hbm_l);
  const bool dev_p = vp != nullptr, dev_l = vl != nullptr;
  int32_t* op = dev_p ? vp : ws->out_parent;
  int32_t* ol = dev_l ? vl : ws->out_level;
  const bool aligned = (((uintptr_t)op | (uintptr_t)ol) & 15) == 0;
  const bool split_ok = aligned && g->relabelled && hbm_p && hbm_l && ws->plo.bits >= 4 &&
                        nb > 1;
  const bool split = split_ok && o->out_split == 2;
  auto translate = [&](cudaStream_t ts) -> g3_status {
    if (split) {
      const int grid = cap_grid((g->n + 3) / 4, 256, ws->grid_tr4);
      bfs_translate_p1<<<grid, 256, 0, ts>>>(g->n, nb, nb / 2, g->new_of_old, ws->visited,
                                             ws->ctrl, ws->plo, (uint32_t*)op);
      G3_CHECK_LAUNCH();
      bfs_translate_p2<<<grid, 256, 0, ts>>>(g->n, root, ws->plo, op, ol);
    } else if (aligned) {
      bfs_translate4<<<cap_grid((g->n + 3) / 4, 256, ws->grid_tr4), 256, 0, ts>>>(
          g->n, nb, root, g->relabelled ? g->new_of_old : nullptr, ws->visited, ws->ctrl,
          ws->plo, op, ol);
    } else {  // outputs not 16-byte aligned
      bfs_translate<<<cap_grid(g->n, 256, ws->grid_tr), 256, 0, ts>>>(
          g->n, nb, root, g->relabelled ? g->new_of_old : nullptr, ws->visited, ws->ctrl,
          ws->plo, op, ol);
    }
    G3_CHECK_LAUNCH();
    return G3_OK;
  };
  bool translated = false;
  if (!host_driven) {
    if (!ws->gexec || !same_opts(ws->gopts, *o) || ws->gfull != full_stats)
      G3_TRY(build_graph(S));
    G3_TRY_CUDA(cudaGraphLaunch(ws->gexec, s));
    // the output pass goes right behind the level loop, without waiting for
    // the host to read the controller; it is repeated below in the rare case
    // of a search deeper than one graph launch runs
    G3_TRY(translate(s));
    translated = true;
  }
  // Host-driven levels: everything in host-driven mode, and what a graph
  // launch left over (searches deeper than its level cap).
  for (;;) {
    G3_TRY_CUDA(cudaMemcpyAsync(h, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    G3_TRY_CUDA(cudaStreamSynchronize(s));
    const int32_t L = h->level;
    if (host_driven && o->timing && L > 0 && stats && L - 1 < max_stats) {
      cudaEventElapsedTime(&stats[L - 1].ms, ws->ev[0], ws->ev[3]);
      cudaEventElapsedTime(&stats[L - 1].ms_expand, ws->ev[1], ws->ev[2]);
    }
    if (h->err) {
      g3_set_error("g3_bfs: a bottom-up kernel's wait for its staged tile ran out");
      return G3_ETIMEOUT;
    }
    if (h->mode == MODE_DONE) break;
    translated = false;
    const int mode = h->mode;
    if (o->record_both && stats && L < max_stats)
      G3_TRY(record_trials(S, h->nf, &stats[L], s));
    if (o->timing) G3_TRY_CUDA(cudaEventRecord(ws->ev[0], s));
    G3_TRY(launch_level(S, mode, h->nf, o->timing ? ws->ev[1] : nullptr, s));
    if (o->timing) G3_TRY_CUDA(cudaEventRecord(ws->ev[2], s));
    CtrlArgs ca = ctrl_args(S, 0, 0, 0);
    bfs_control<<<1, 32, 0, s>>>(ws->ctrl, ca);
    G3_CHECK_LAUNCH();
    if (o->timing) G3_TRY_CUDA(cudaEventRecord(ws->ev[3], s));
  }
  const int32_t nrec = h->level;  // non-empty frontiers F_0 .. F_{nrec-1}
  if (n_levels) *n_levels = nrec;

  if (!translated) G3_TRY(translate(s));
  if (!dev_p)
    G3_TRY_CUDA(cudaMemcpyAsync(parent, op, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
  if (!dev_l)
    G3_TRY_CUDA(cudaMemcpyAsync(level, ol, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
  // per-level records from the device log
  const int32_t nlog = nrec < LOG_MAX ? nrec : LOG_MAX;
  const int32_t ncopy = stats ? (nlog < max_stats ? nlog : max_stats) : 0;
  LevelLog* hl = nullptr;
  if (ncopy > 0) {
    hl = (LevelLog*)malloc(sizeof(LevelLog) * (size_t)ncopy);
    if (!hl) return G3_ENOMEM;
    cudaError_t e =
        cudaMemcpyAsync(hl, ws->log, sizeof(LevelLog) * (size_t)ncopy, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
      free(hl);
      G3_TRY_CUDA(e);
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess)
    for (int32_t L = 0; L < ncopy; ++L) fill_record(&stats[L], L, hl[L]);
  free(hl);
  G3_TRY_CUDA(e);
  return G3_OK;
}

g3_status g3_bfs_multi_root(g3_graph* g, const int32_t* roots, int32_t count, const int32_t* lo,
                            const g3_bfs_opts* opts, int32_t* parent, int32_t* level,
                            cudaStream_t s) {
  g3_bfs_opts o;
  if (opts) o = *opts; else g3_bfs_opts_default(&o);
  MultiRoots mr{roots, count, lo};
  g3_status st = bfs_impl(g, -1, &o, parent, level, nullptr, 0, nullptr, s, &mr);
  if (st != G3_OK) cudaStreamSynchronize(s);
  return st;
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
      o.t2 <= o.t1 || o.t3 <= o.t2 || o.mlp_margin < 0 || o.out_split < 0 || o.out_split > 2 ||
      o.bu_kernel < 0 || o.bu_kernel > 3) {
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
