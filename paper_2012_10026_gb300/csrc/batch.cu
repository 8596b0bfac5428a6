// Batched BFS over many small graphs in one persistent launch (no
// counterpart in the paper, which searches one graph at a time).
//
// g3_batch_pack concatenates already relabelled graphs into one union CSR
// (graph g keeps the vertex range [voff[g], voff[g+1]) in both ID spaces).
// Two ways to search the batch (g3_batch_opts.mode):
//  0  one persistent kernel per launch, captured once into a CUDA graph
// together with the reset of its work counters: resident blocks take graphs
// from two work lists with an atomic counter -- graphs with at most
// warp_max_n BFS vertices are searched by one warp each, larger ones by a
// whole CTA -- and each group keeps its graph's visited, current and next
// frontier bitmaps in shared memory. Every level is expanded top-down (warp
// per frontier vertex, lanes over its neighbours, shared-memory atomicOr
// claims) or bottom-up (lane per vertex, early exit on the first frontier
// neighbour), chosen by the same alpha/beta rule as g3_bfs; parent[] and
// level[] are written in original IDs inside the graph's own ID range.
//  1  one level-synchronous search over the whole union, seeded with every
//     graph's root at once: the graphs are disjoint, so no level of one can
//     reach another, and the single-source machinery (degree-binned top-down,
//     bottom-up pull, device controller, level loop as a CUDA graph) runs
//     over all of them with the whole GPU behind every level.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "g3_internal.cuh"

#define BT_CTA_WORDS 512  // CTA groups: up to 16384 BFS vertices per graph
#define BT_WARP_WORDS 64  // warp groups: up to 2048 BFS vertices per graph

struct g3_batch {
  int32_t G;
  int64_t N, nnz;
  int64_t* off;  // [N+1]
  int32_t* col;  // [nnz], union labels
  int32_t* orig_of;   // [N] union label -> union original ID
  int32_t* label_of;  // [N] union original ID -> union label
  int32_t* voff; // [G+1]
  int32_t* np;   // [G] BFS vertices per graph (V+)
  int32_t* order_warp;
  int32_t* order_cta;
  unsigned* counters;  // [2]
  std::vector<int32_t> h_voff, h_np;
  // captured launch
  cudaGraphExec_t gexec;
  const int32_t* g_roots;
  int32_t *g_parent, *g_level;
  int32_t g_thresh;
  int32_t n_warp, n_cta;
  cudaEvent_t ev[2];
  g3_graph ug;  // the union as a relabelled graph (arrays above, not owned)
};

struct BatchArgs {
  int64_t N;
  const int64_t* off;
  const int32_t* col;
  const int32_t* orig_of;
  const int32_t* label_of;
  const int32_t* voff;
  const int32_t* np;
  const int32_t* roots;
  int32_t* parent;
  int32_t* level;
};

// Group-wide barrier: a warp group needs only the warp.
template <int GT>
__device__ __forceinline__ void group_sync() {
  if (GT == 32) __syncwarp(); else __syncthreads();
}

// One BFS of graph g by a group of GT threads (a warp or the whole CTA) with
// the graph's bitmaps in shared memory: bm = visited, current and next
// frontier, MAXW words each; s_cnt = two group-shared counters.
template <int GT, int MAXW>
__device__ __forceinline__ void batch_search(const BatchArgs& A, int32_t g, uint32_t* bm,
                                             unsigned long long* s_cnt, int t) {
  constexpr int WPG = GT / 32;  // warps per group
  const int lane = threadIdx.x & 31, wig = t >> 5;
  uint32_t* vis = bm;
  uint32_t* cur = bm + MAXW;
  uint32_t* nxt = bm + 2 * MAXW;
  const int32_t vb = A.voff[g], ng = A.voff[g + 1] - vb, npg = A.np[g];
  const int32_t words = (npg + 31) >> 5;
  const int32_t root_o = A.roots[g];
  // a root outside its own graph's ID range leaves the graph unreached
  const bool root_ok = root_o >= vb && root_o < vb + ng;
  const int32_t r = root_ok ? A.label_of[root_o] - vb : npg;
  for (int32_t i = t; i < ng; i += GT) {
    A.parent[vb + i] = -1;
    A.level[vb + i] = -1;
  }
  for (int32_t w = t; w < words; w += GT) {
    vis[w] = 0u;
    cur[w] = 0u;
  }
  group_sync<GT>();
  if (t == 0 && root_ok) {
    A.parent[root_o] = root_o;
    A.level[root_o] = 0;
    if (r >= 0 && r < npg) {
      vis[r >> 5] |= 1u << (r & 31);
      cur[r >> 5] |= 1u << (r & 31);
    }
  }
  group_sync<GT>();
  if (r < 0 || r >= npg) return;  // isolated root: nothing else is reached
  const int64_t mtot = A.off[vb + npg] - A.off[vb];
  int64_t mvis = A.off[vb + r + 1] - A.off[vb + r];
  int64_t mf = mvis, prev_nf = 0, nf = 1;
  bool bu = false;
  for (int32_t L = 0;; ++L) {
    // direction for this level (Algorithm 2 starts top-down; alpha/beta rule)
    if (L > 0) {
      const int64_t mu = mtot - mvis;
      bu = bu ? !(nf < prev_nf && nf * 24 < npg) : (mf * 14 > mu);
    }
    for (int32_t w = t; w < words; w += GT) nxt[w] = 0u;
    if (t == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
    }
    group_sync<GT>();
    unsigned long long cnt = 0, dsum = 0;
    if (!bu) {
      // top-down: each warp takes frontier words, the whole warp expands
      // each frontier vertex of the word
      for (int32_t w = wig; w < words; w += WPG) {
        uint32_t bits = cur[w];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1u;
          const int32_t V = vb + w * 32 + b;
          const int32_t vo = A.orig_of[V];
          const int64_t e = A.off[V + 1];
          for (int64_t j = A.off[V] + lane; j < e; j += 32) {
            const int32_t u = A.col[j] - vb;
            const uint32_t bit = 1u << (u & 31);
            if (!(vis[u >> 5] & bit) && !(atomicOr(&vis[u >> 5], bit) & bit)) {
              atomicOr(&nxt[u >> 5], bit);
              const int32_t uo = A.orig_of[vb + u];
              A.parent[uo] = vo;
              A.level[uo] = L + 1;
              cnt++;
              dsum += (unsigned long long)(A.off[vb + u + 1] - A.off[vb + u]);
            }
          }
        }
      }
    } else {
      // bottom-up: lane per vertex, scan from the row's end (highest label
      // first), stop at the first neighbour in the current frontier
      for (int32_t w = wig; w < words; w += WPG) {
        const int32_t v = w * 32 + lane;
        const bool cand = v < npg && !((vis[w] >> lane) & 1u);
        int32_t p = -1;
        int64_t d = 0;
        if (cand) {
          const int64_t b0 = A.off[vb + v], e0 = A.off[vb + v + 1];
          d = e0 - b0;
          for (int64_t j = e0 - 1; j >= b0; --j) {
            const int32_t u = A.col[j] - vb;
            if ((cur[u >> 5] >> (u & 31)) & 1u) {
              p = u;
              break;
            }
          }
        }
        const uint32_t found = __ballot_sync(0xffffffffu, p >= 0);
        if (lane == 0 && found) {
          nxt[w] = found;
          vis[w] |= found;
        }
        if (p >= 0) {
          const int32_t vo = A.orig_of[vb + v];
          A.parent[vo] = A.orig_of[vb + p];
          A.level[vo] = L + 1;
          cnt++;
          dsum += (unsigned long long)d;
        }
      }
    }
    for (int o = 16; o; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    }
    if (lane == 0 && cnt) {
      atomicAdd(&s_cnt[0], cnt);
      atomicAdd(&s_cnt[1], dsum);
    }
    group_sync<GT>();
    prev_nf = nf;
    nf = (int64_t)s_cnt[0];
    mf = (int64_t)s_cnt[1];
    mvis += mf;
    uint32_t* tmp = cur;
    cur = nxt;
    nxt = tmp;
    group_sync<GT>();
    if (nf == 0) break;
  }
}

// Persistent kernel over all graphs, 512 threads per CTA: first every CTA
// takes graphs of the CTA list (largest first) as a whole, then, once that
// list is drained, each warp takes graphs of the warp list on its own; the
// tail of the big graphs overlaps the small ones. counters[0] / [1] are the
// two lists' cursors. (512-thread CTAs halve each big graph's per-thread
// chains against 256 at the same occupancy.)
__global__ void __launch_bounds__(512) batch_bfs(BatchArgs A, const int32_t* __restrict__ order_cta,
                                                 int32_t n_cta,
                                                 const int32_t* __restrict__ order_warp,
                                                 int32_t n_warp, unsigned* counters) {
  __shared__ uint32_t bm[16 * 3 * BT_WARP_WORDS];
  __shared__ unsigned long long s_cnt[16][2];
  __shared__ int s_gi[16];
  for (;;) {
    if (threadIdx.x == 0) s_gi[0] = (int)atomicAdd(&counters[0], 1u);
    __syncthreads();
    const int gi = s_gi[0];
    __syncthreads();
    if (gi >= n_cta) break;
    batch_search<512, BT_CTA_WORDS>(A, order_cta[gi], bm, s_cnt[0], threadIdx.x);
    __syncthreads();
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* wbm = bm + wid * 3 * BT_WARP_WORDS;
  for (;;) {
    int gi = 0;
    if (lane == 0) gi = (int)atomicAdd(&counters[1], 1u);
    gi = __shfl_sync(0xffffffffu, gi, 0);
    if (gi >= n_warp) break;
    batch_search<32, BT_WARP_WORDS>(A, order_warp[gi], wbm, s_cnt[wid], lane);
    __syncwarp();
  }
}

// Copies one graph's relabelled CSR (n rows) into the union, shifted to its
// vertex and edge ranges.
__global__ void batch_shift(const int64_t* __restrict__ off_in, const int32_t* __restrict__ col_in,
                            int32_t n, int64_t nnz, int32_t vb, int64_t eb, int64_t* off_out,
                            int32_t* col_out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz || i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nnz) col_out[i] = col_in[i] + vb;
    if (i < n) off_out[i] = off_in[i] + eb;
  }
}

// ------------------------------------------------------------------ host
extern "C" void g3_batch_free(g3_batch* b) {
  if (!b) return;
  void* all[] = {b->off, b->col, b->orig_of, b->label_of, b->voff, b->np, b->order_warp, b->order_cta,
                 b->counters};
  for (void* p : all)
    if (p) cudaFree(p);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (int i = 0; i < 2; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  g3_bfs_ws_free(b->ug.ws);
  delete b;
}

extern "C" g3_status g3_batch_pack(g3_graph* const* graphs, int32_t G, void* stream,
                                   g3_batch** out) {
  if (!out || !graphs || G <= 0) {
    g3_set_error("g3_batch_pack: bad arguments");
    return G3_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t N = 0, nnz = 0, maxdeg = 0;
  for (int32_t i = 0; i < G; ++i) {
    const g3_graph* g = graphs[i];
    if (!g || !g->relabelled) {
      g3_set_error("g3_batch_pack: graph %d is missing or not relabelled", i);
      return G3_EINVAL;
    }
    if (g->n_plus > BT_CTA_WORDS * 32) {
      g3_set_error("g3_batch_pack: graph %d has %d BFS vertices (limit %d)", i, g->n_plus,
                   BT_CTA_WORDS * 32);
      return G3_EINVAL;
    }
    N += g->n;
    nnz += g->nnz;
    maxdeg = std::max<int64_t>(maxdeg, g->max_degree);
  }
  if (N >= (1ll << 31)) {
    g3_set_error("g3_batch_pack: %lld vertices in total do not fit int32", (long long)N);
    return G3_EINVAL;
  }
  g3_batch* b = new g3_batch();
  b->G = G;
  b->N = N;
  b->nnz = nnz;
  g3_status st = G3_OK;
  struct {
    void** p;
    size_t bytes;
  } req[] = {{(void**)&b->off, (size_t)(N + 1) * 8},  {(void**)&b->col, (size_t)nnz * 4 + 16},
             {(void**)&b->orig_of, (size_t)N * 4 + 16},   {(void**)&b->label_of, (size_t)N * 4 + 16},
             {(void**)&b->voff, (size_t)(G + 1) * 4}, {(void**)&b->np, (size_t)G * 4},
             {(void**)&b->order_warp, (size_t)G * 4}, {(void**)&b->order_cta, (size_t)G * 4},
             {(void**)&b->counters, 16}};
  for (auto& r : req) {
    if (g3_alloc_should_fail() || cudaMalloc(r.p, r.bytes) != cudaSuccess) {
      cudaGetLastError();
      g3_set_error("g3_batch_pack: cudaMalloc(%zu) failed", r.bytes);
      g3_batch_free(b);
      return G3_ENOMEM;
    }
  }
  if (cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
    cudaGetLastError();
    g3_batch_free(b);
    return G3_ECUDA;
  }
  b->h_voff.resize(G + 1);
  b->h_np.resize(G);
  int64_t vb = 0, eb = 0;
  for (int32_t i = 0; i < G && st == G3_OK; ++i) {
    const g3_graph* g = graphs[i];
    b->h_voff[i] = (int32_t)vb;
    b->h_np[i] = g->n_plus;
    // the relabelled CSR has n_plus rows; the isolated vertices of the graph
    // (labels n_plus .. n-1) get empty rows
    batch_shift<<<g3_grid_for(std::max<int64_t>(g->nnz, g->n_plus), 256), 256, 0, s>>>(
        g->off, g->col, g->n_plus, g->nnz, (int32_t)vb, eb, b->off + vb, b->col + eb);
    g3_count_launch();
    if (cudaGetLastError() != cudaSuccess) st = G3_ECUDA;
    if (g->n > g->n_plus) {
      // rows of isolated vertices start (and end) at the graph's last offset
      std::vector<int64_t> tail((size_t)(g->n - g->n_plus), eb + g->nnz);
      if (cudaMemcpy(b->off + vb + g->n_plus, tail.data(), tail.size() * 8,
                     cudaMemcpyHostToDevice) != cudaSuccess)
        st = G3_ECUDA;
    }
    vb += g->n;
    eb += g->nnz;
  }
  b->h_voff[G] = (int32_t)vb;
  if (st == G3_OK) {
    // union label maps: graph g's labels and original IDs both shifted by
    // its vertex offset
    std::vector<int32_t> orig_of((size_t)N), label_of((size_t)N);
    int64_t base = 0;
    cudaStreamSynchronize(s);
    for (int32_t i = 0; i < G && st == G3_OK; ++i) {
      const g3_graph* g = graphs[i];
      if (cudaMemcpy(orig_of.data() + base, g->old_of_new, (size_t)g->n * 4,
                     cudaMemcpyDeviceToHost) != cudaSuccess)
        st = G3_ECUDA;
      for (int32_t v = 0; v < g->n; ++v) {
        orig_of[base + v] += (int32_t)base;
        label_of[orig_of[base + v]] = (int32_t)(base + v);
      }
      base += g->n;
    }
    if (st == G3_OK) {
      if (cudaMemcpy(b->orig_of, orig_of.data(), (size_t)N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(b->label_of, label_of.data(), (size_t)N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(b->off + N, &nnz, 8, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(b->voff, b->h_voff.data(), (size_t)(G + 1) * 4, cudaMemcpyHostToDevice) !=
              cudaSuccess ||
          cudaMemcpy(b->np, b->h_np.data(), (size_t)G * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        st = G3_ECUDA;
    }
  }
  if (st != G3_OK) {
    g3_set_error("g3_batch_pack: copy failed");
    g3_batch_free(b);
    return st;
  }
  b->g_thresh = -1;
  // the union as one relabelled graph: every union vertex is a BFS-graph
  // vertex (isolated ones have empty rows)
  b->ug.n = (int32_t)N;
  b->ug.nnz = nnz;
  b->ug.max_degree = maxdeg;
  b->ug.n_bfs = (int32_t)N;
  b->ug.n_plus = (int32_t)N;
  b->ug.relabelled = 1;
  b->ug.off = b->off;
  b->ug.col = b->col;
  b->ug.old_of_new = b->orig_of;
  b->ug.new_of_old = b->label_of;
  *out = b;
  return G3_OK;
}

extern "C" void g3_batch_opts_default(g3_batch_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->warp_max_n = 1024;
  o->mode = 0;
}

extern "C" g3_status g3_batch_info_get(const g3_batch* b, int32_t* G, int64_t* N, int64_t* nnz) {
  if (!b) {
    g3_set_error("g3_batch_info_get: batch is NULL");
    return G3_EINVAL;
  }
  if (G) *G = b->G;
  if (N) *N = b->N;
  if (nnz) *nnz = b->nnz;
  return G3_OK;
}

// (Re)captures the launch: counter reset, warp-group kernel, CTA-group kernel.
static g3_status batch_capture(g3_batch* b, const int32_t* roots, int32_t* parent,
                               int32_t* level, int32_t thresh) {
  std::vector<int32_t> warp_list, cta_list;
  for (int32_t g = 0; g < b->G; ++g)
    (b->h_np[g] <= thresh && b->h_np[g] <= BT_WARP_WORDS * 32 ? warp_list : cta_list).push_back(g);
  // largest graphs first so the tail of the persistent loop is short
  auto by_size = [&](int32_t x, int32_t y) { return b->h_np[x] > b->h_np[y]; };
  std::sort(warp_list.begin(), warp_list.end(), by_size);
  std::sort(cta_list.begin(), cta_list.end(), by_size);
  if (!warp_list.empty())
    G3_TRY_CUDA(cudaMemcpy(b->order_warp, warp_list.data(), warp_list.size() * 4,
                           cudaMemcpyHostToDevice));
  if (!cta_list.empty())
    G3_TRY_CUDA(cudaMemcpy(b->order_cta, cta_list.data(), cta_list.size() * 4,
                           cudaMemcpyHostToDevice));
  b->n_warp = (int32_t)warp_list.size();
  b->n_cta = (int32_t)cta_list.size();
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_bfs, 512, 0);
  const int grid =
      std::max(1, std::min(sms * std::max(per, 1), std::max(b->n_cta, (b->n_warp + 15) / 16)));
  BatchArgs A{b->N, b->off, b->col, b->orig_of, b->label_of, b->voff, b->np, roots, parent, level};
  cudaStream_t cs;
  G3_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(b->counters, 0, 16, cs);
    batch_bfs<<<grid, 512, 0, cs>>>(A, b->order_cta, b->n_cta, b->order_warp, b->n_warp,
                                    b->counters);
  e = cudaStreamEndCapture(cs, &graph);
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g3_set_error("g3_bfs_batch: capture failed: %s", cudaGetErrorString(e));
    return G3_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g3_set_error("g3_bfs_batch: instantiate failed: %s", cudaGetErrorString(e));
    return G3_ECUDA;
  }
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = ex;
  b->g_roots = roots;
  b->g_parent = parent;
  b->g_level = level;
  b->g_thresh = thresh;
  return G3_OK;
}

extern "C" g3_status g3_bfs_batch(g3_batch* b, const int32_t* roots, const g3_batch_opts* opts,
                                  int32_t* parent, int32_t* level, float* ms, void* stream) {
  if (!b || !roots || !parent || !level) {
    g3_set_error("g3_bfs_batch: null argument");
    return G3_EINVAL;
  }
  g3_batch_opts o;
  if (opts) o = *opts; else g3_batch_opts_default(&o);
  if (o.warp_max_n < 0 || o.mode < 0 || o.mode > 1) {
    g3_set_error("g3_bfs_batch: bad options");
    return G3_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (o.mode == 1) {
    G3_TRY_CUDA(cudaEventRecord(b->ev[0], s));
    G3_TRY(g3_bfs_multi_root(&b->ug, roots, b->G, b->voff, nullptr, parent, level, s));
    G3_TRY_CUDA(cudaEventRecord(b->ev[1], s));
    if (ms) {
      G3_TRY_CUDA(cudaEventSynchronize(b->ev[1]));
      cudaEventElapsedTime(ms, b->ev[0], b->ev[1]);
    }
    return G3_OK;
  }
  if (!b->gexec || b->g_roots != roots || b->g_parent != parent || b->g_level != level ||
      b->g_thresh != o.warp_max_n) {
    G3_TRY_CUDA(cudaStreamSynchronize(s));
    G3_TRY(batch_capture(b, roots, parent, level, o.warp_max_n));
  }
  G3_TRY_CUDA(cudaEventRecord(b->ev[0], s));
  G3_TRY_CUDA(cudaGraphLaunch(b->gexec, s));
  g3_count_launch();
  G3_TRY_CUDA(cudaEventRecord(b->ev[1], s));
  if (ms) {
    G3_TRY_CUDA(cudaEventSynchronize(b->ev[1]));
    cudaEventElapsedTime(ms, b->ev[0], b->ev[1]);
  }
  return G3_OK;
}
