// Reverse Cuthill-McKee relabelling, Algorithm 3 (Sec. 3.2), computed
// level-synchronously on the GPU and equal to the serial algorithm:
//
//  1. V+ (degree > 0) sorted by (degree, ID): rank[v] = position in V+.
//  2. Connected components in rank space by min-hooking and pointer jumping;
//     every tree root is the smallest rank of its component, i.e. the vertex
//     Algorithm 3 starts that component from (the first unvisited vertex of
//     V+), and components are taken in order of that rank.
//  3. Component c owns Cuthill-McKee positions [base_c, base_c + |c|)
//     (exclusive scan of the sizes in rank order); its start gets base_c.
//  4. All components advance together, one BFS level per step. A vertex w
//     first reached from level k gets ppos[w] = the smallest CM position of
//     its neighbours in level k (atomicMin). The queue of Algorithm 3 appends
//     the neighbours of each level-k vertex, in (degree, ID) order, when that
//     vertex is dequeued, so level k+1 of a component comes out ordered by
//     (ppos, degree, ID) = (ppos, rank). One radix sort of the level by that
//     key, then each component's slice takes the next positions of its range.
//  5. Reverse: label = n_plus - 1 - position; isolated vertices get n_plus..n-1
//     in ascending ID. The CSR is rebuilt under the new labels (rows sorted).
//
// Partial RCM (Sec. 4.6) runs the same steps on S = the vertices of rank >= lo
// only (the top k of V+ by (degree, ID), lo = n_plus - k): edges leaving S are
// ignored by the hooking and the level expansion, S takes labels k-1-position,
// and the rest of V+ takes labels k.. in ascending ID. lo = 0 is the full
// algorithm.
#include "g3_prims.cuh"

#define INF_U32 0xFFFFFFFFu

// ------------------------------------------------------------ V+ and ranks
struct IsNonIsolated {
  const int64_t* off;
  __device__ bool operator()(int64_t v) const { return off[v + 1] > off[v]; }
};
struct EmitDegKey {
  const int64_t* off;
  uint64_t* keys;
  int bits_v;
  __device__ void operator()(int64_t v, int64_t pos) const {
    keys[pos] = ((uint64_t)(off[v + 1] - off[v]) << bits_v) | (uint64_t)v;
  }
};
struct IsIsolated {
  const int64_t* off;
  __device__ bool operator()(int64_t v) const { return off[v + 1] == off[v]; }
};
struct EmitIsolatedLabel {
  int32_t n_plus;
  int32_t* new_of_old;
  __device__ void operator()(int64_t v, int64_t pos) const {
    new_of_old[v] = n_plus + (int32_t)pos;
  }
};

__global__ void rcm_ranks(const uint64_t* __restrict__ keys, int32_t n_plus, int bits_v,
                          int32_t* __restrict__ vplus, int32_t* __restrict__ rank,
                          int32_t* __restrict__ parent) {
  const uint64_t mask = (1ull << bits_v) - 1ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_plus;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = (int32_t)(keys[r] & mask);
    vplus[r] = v;
    rank[v] = (int32_t)r;
    parent[r] = (int32_t)r;
  }
}

// --------------------------------------------------------------- components
__device__ __forceinline__ int32_t uf_find(const int32_t* p, int32_t r) {
  int32_t q = __ldcg(&p[r]);
  while (q != r) {
    r = q;
    q = __ldcg(&p[r]);
  }
  return r;
}

struct HookEdge {
  const int32_t* col;
  const int32_t* rank;
  int32_t* p;
  int* changed;
  int32_t lo;  // only edges inside ranks [lo, n_plus)
  __device__ void operator()(int64_t u, int64_t j, bool active) const {
    if (!active) return;
    int32_t w = col[j];
    if ((int32_t)u >= w) return;  // each undirected edge once
    if (rank[u] < lo || rank[w] < lo) return;
    int32_t ru = uf_find(p, rank[u]), rw = uf_find(p, rank[w]);
    if (ru == rw) return;
    int32_t lo = ru < rw ? ru : rw, hi = ru < rw ? rw : ru;
    atomicMin(&p[hi], lo);
    *changed = 1;
  }
};

__global__ void __launch_bounds__(256) rcm_hook(const int64_t* off, int32_t n, HookEdge f) {
  g3_for_each_entry(off, n, f);
}

__global__ void rcm_compress(int32_t* p, int32_t n_plus) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_plus;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t root = uf_find(p, (int32_t)r);
    p[r] = root;
  }
}

// Component sizes, warp-aggregated per distinct root.
__global__ void rcm_comp_sizes(const int32_t* __restrict__ p, int32_t n_plus, int32_t lo,
                               unsigned long long* size) {
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n_plus;
       base += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = base + threadIdx.x;
    int32_t root = (r < n_plus && r >= lo) ? p[r] : -1;
    unsigned peers = __match_any_sync(0xffffffffu, root);
    if (root >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
      atomicAdd(&size[root], (unsigned long long)__popc(peers));
  }
}

struct IsRoot {
  const int32_t* p;
  int32_t lo;
  __device__ bool operator()(int64_t r) const { return r >= lo && p[r] == (int32_t)r; }
};
struct EmitStart {
  const int32_t* vplus;
  const int64_t* base;
  int32_t* pos;
  int64_t* cursor;
  int32_t* front;
  __device__ void operator()(int64_t r, int64_t i) const {
    int32_t v = vplus[r];
    pos[v] = (int32_t)base[r];
    cursor[r] = base[r] + 1;
    front[i] = v;
  }
};

// ------------------------------------------------------------- level steps
__global__ void rcm_front_degrees(const int32_t* __restrict__ front, int64_t nf,
                                  const int64_t* __restrict__ off, int64_t* fdeg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = front[i];
    fdeg[i] = off[v + 1] - off[v];
  }
}

struct ExpandLevel {
  const int32_t* front;
  const int64_t* fseg;
  const int64_t* off;
  const int32_t* col;
  const int32_t* pos;
  uint32_t* ppos;
  int32_t* next;
  unsigned long long* next_len;
  const int32_t* rank;
  int32_t lo;
  __device__ void operator()(int64_t i, int64_t j, bool active) const {
    bool claim = false;
    int32_t w = 0;
    if (active) {
      int32_t v = front[i];
      w = col[off[v] + (j - fseg[i])];
      if (pos[w] < 0 && rank[w] >= lo) {
        uint32_t old = atomicMin(&ppos[w], (uint32_t)pos[v]);
        claim = old == INF_U32;
      }
    }
    g3_warp_append(0xffffffffu, claim, w, next, next_len);
  }
};

__global__ void __launch_bounds__(256) rcm_expand(const int64_t* fseg, int64_t nf, ExpandLevel f) {
  g3_for_each_entry(fseg, nf, f);
}

__global__ void rcm_level_keys(const int32_t* __restrict__ next, int64_t len,
                               const uint32_t* __restrict__ ppos,
                               const int32_t* __restrict__ rank, int bits_r,
                               uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t w = next[i];
    keys[i] = ((uint64_t)ppos[w] << bits_r) | (uint64_t)rank[w];
  }
}

// component (root rank) of sorted element i
__device__ __forceinline__ int32_t comp_of(const uint64_t* keys, int64_t i, uint64_t mask,
                                           const int32_t* p) {
  return p[(int32_t)(keys[i] & mask)];
}

__global__ void rcm_level_heads(const uint64_t* __restrict__ keys, int64_t len, int bits_r,
                                const int32_t* __restrict__ p, int64_t* first) {
  const uint64_t mask = (1ull << bits_r) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = comp_of(keys, i, mask, p);
    if (i == 0 || comp_of(keys, i - 1, mask, p) != c) first[c] = i;
  }
}

__global__ void rcm_level_place(const uint64_t* __restrict__ keys, int64_t len, int bits_r,
                                const int32_t* __restrict__ p,
                                const int32_t* __restrict__ vplus,
                                const int64_t* __restrict__ first,
                                const int64_t* __restrict__ cursor, int32_t* pos,
                                int32_t* front) {
  const uint64_t mask = (1ull << bits_r) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = (int32_t)(keys[i] & mask);
    int32_t c = p[r];
    int32_t w = vplus[r];
    pos[w] = (int32_t)(cursor[c] + (i - first[c]));
    front[i] = w;
  }
}

__global__ void rcm_level_tails(const uint64_t* __restrict__ keys, int64_t len, int bits_r,
                                const int32_t* __restrict__ p,
                                const int64_t* __restrict__ first, int64_t* cursor) {
  const uint64_t mask = (1ull << bits_r) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = comp_of(keys, i, mask, p);
    if (i == len - 1 || comp_of(keys, i + 1, mask, p) != c) cursor[c] += i - first[c] + 1;
  }
}

// ------------------------------------------------------------- relabel CSR
__global__ void rcm_labels(const int32_t* __restrict__ pos, int32_t n, int32_t k,
                           int32_t* new_of_old) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t q = pos[v];
    if (q >= 0) new_of_old[v] = k - 1 - q;
  }
}

// Label range of each vertex's component (full relabelling). The component
// started from rank c holds Cuthill-McKee positions [base[c], cursor[c])
// once every level is placed, and the reversal turns position q into label
// k - 1 - q, so its labels are [k - cursor[c], k - base[c]).
__global__ void rcm_comp_ranges(const int32_t* __restrict__ rank, const int32_t* __restrict__ p,
                                const int64_t* __restrict__ base,
                                const int64_t* __restrict__ cursor,
                                const int32_t* __restrict__ new_of_old, int32_t n, int32_t k,
                                int2* rng) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rank[v];
    if (r < 0) continue;  // isolated
    const int32_t c = p[r];
    rng[new_of_old[v]] = make_int2(k - (int32_t)cursor[c], k - (int32_t)base[c]);
  }
}

// Partial RCM: the vertices of V+ below rank lo, labels k.. by ascending ID.
struct IsUnordered {
  const int64_t* off;
  const int32_t* rank;
  int32_t lo;
  __device__ bool operator()(int64_t v) const { return off[v + 1] > off[v] && rank[v] < lo; }
};
struct EmitUnorderedLabel {
  int32_t k;
  int32_t* new_of_old;
  __device__ void operator()(int64_t v, int64_t pos) const {
    new_of_old[v] = k + (int32_t)pos;
  }
};

__global__ void rcm_inverse(const int32_t* __restrict__ new_of_old, int32_t n,
                            const int64_t* __restrict__ off, int32_t* old_of_new,
                            int64_t* deg_new) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t l = new_of_old[v];
    old_of_new[l] = (int32_t)v;
    int64_t d = off[v + 1] - off[v];
    if (d > 0) deg_new[l] = d;
  }
}

struct PermKey {
  const int32_t* col;
  const int32_t* new_of_old;
  uint64_t* keys;
  int bits;
  __device__ void operator()(int64_t u, int64_t j, bool active) const {
    if (!active) return;
    keys[j] = ((uint64_t)new_of_old[u] << bits) | (uint64_t)new_of_old[col[j]];
  }
};

__global__ void __launch_bounds__(256) rcm_perm_keys(const int64_t* off, int32_t n, PermKey f) {
  g3_for_each_entry(off, n, f);
}

__global__ void rcm_take_col(const uint64_t* __restrict__ keys, int64_t nnz, int bits,
                             int32_t* __restrict__ col) {
  const uint64_t mask = (1ull << bits) - 1ull;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x)
    col[j] = (int32_t)(keys[j] & mask);
}

// ---------------------------------------------------------------- driver
static g3_status read_i64(const int64_t* d, int64_t* h, cudaStream_t s) {
  G3_TRY_CUDA(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  return G3_OK;
}

extern "C" g3_status g3_graph_max_degree(g3_graph* g, cudaStream_t s);

struct RcmBufs {
  uint64_t *ka = nullptr, *kb = nullptr;
  int64_t* partial = nullptr;
  int32_t *vplus = nullptr, *rank = nullptr, *p = nullptr, *pos = nullptr;
  uint32_t* ppos = nullptr;
  int64_t *base = nullptr, *cursor = nullptr, *first = nullptr, *fseg = nullptr;
  int32_t *front = nullptr, *next = nullptr;
  unsigned long long* counters = nullptr;  // [0]=changed (int), [1]=next_len
  int64_t* deg_new = nullptr;
  void release(cudaStream_t s) {
    void* all[] = {ka, kb, partial, vplus, rank, p, pos, ppos, base, cursor, first,
                   fseg, front, next, counters, deg_new};
    for (void* x : all) g3_free(x, s);
  }
};

static g3_status rcm_impl(g3_graph* g, int32_t p_permille, cudaStream_t s, RcmBufs& B) {
  const int32_t n = g->n;
  const int64_t nnz = g->nnz;
  const int bits_v = g3_bits_for(n);
  const int grid = G3_NUM_SMS * 8;
  G3_TRY(g3_alloc(&B.partial, g3_compact_partials(n) + 4, s));
  G3_TRY(g3_alloc(&B.ka, n, s));
  G3_TRY(g3_alloc(&B.kb, n, s));
  g3_free(g->new_of_old, s);
  g3_free(g->old_of_new, s);
  g3_free(g->comp_rng, s);
  g->new_of_old = g->old_of_new = nullptr;
  g->comp_rng = nullptr;
  G3_TRY(g3_alloc(&g->new_of_old, n, s));
  G3_TRY(g3_alloc(&g->old_of_new, n, s));
  G3_TRY(g3_alloc(&B.counters, 2, s));

  // 1. V+ by (degree, ID)
  G3_TRY(g3_compact((int64_t)n, IsNonIsolated{g->off}, EmitDegKey{g->off, B.ka, bits_v},
                    B.partial, s));
  int64_t nplus64 = 0;
  G3_TRY(read_i64(B.partial + (n + CP_TILE - 1) / CP_TILE, &nplus64, s));
  const int32_t n_plus = (int32_t)nplus64;
  // the top k of V+ are reordered (all of it for the full algorithm)
  const int32_t k = (int32_t)(((int64_t)n_plus * p_permille + 999) / 1000);
  const int32_t lo = n_plus - k;
  const int bits_d = g3_bits_for(g->max_degree + 1);
  uint64_t* sorted;
  G3_TRY(g3_radix_sort_u64(B.ka, B.kb, n_plus, bits_d + bits_v, &sorted, s));
  G3_TRY(g3_alloc(&B.vplus, (size_t)n_plus + 1, s));
  G3_TRY(g3_alloc(&B.rank, n, s));
  G3_TRY(g3_alloc(&B.p, (size_t)n_plus + 1, s));
  G3_TRY_CUDA(cudaMemsetAsync(B.rank, 0xFF, (size_t)n * sizeof(int32_t), s));
  if (n_plus > 0) {
    rcm_ranks<<<g3_grid_for(n_plus, 256), 256, 0, s>>>(sorted, n_plus, bits_v, B.vplus, B.rank,
                                                       B.p);
    G3_CHECK_LAUNCH();
  }

  // 2. components (roots = smallest rank of each component)
  for (int it = 0; n_plus > 0; ++it) {
    G3_TRY_CUDA(cudaMemsetAsync(B.counters, 0, sizeof(unsigned long long), s));
    rcm_hook<<<grid, 256, 0, s>>>(g->off, n,
                                  HookEdge{g->col, B.rank, B.p, (int*)B.counters, lo});
    G3_CHECK_LAUNCH();
    rcm_compress<<<g3_grid_for(n_plus, 256), 256, 0, s>>>(B.p, n_plus);
    G3_CHECK_LAUNCH();
    int changed = 0;
    G3_TRY_CUDA(cudaMemcpyAsync(&changed, B.counters, sizeof(int), cudaMemcpyDeviceToHost, s));
    G3_TRY_CUDA(cudaStreamSynchronize(s));
    if (!changed) break;
    if (it >= g3_rcm_hook_cap()) {
      g3_set_error("g3_rcm_relabel: component hooking did not converge");
      return G3_ETIMEOUT;
    }
  }

  // 3. component position ranges, starts
  G3_TRY(g3_alloc(&B.base, (size_t)n_plus + 1, s));
  G3_TRY(g3_alloc(&B.cursor, (size_t)n_plus + 1, s));
  G3_TRY(g3_alloc(&B.first, (size_t)n_plus + 1, s));
  G3_TRY_CUDA(cudaMemsetAsync(B.base, 0, ((size_t)n_plus + 1) * sizeof(int64_t), s));
  if (n_plus > 0) {
    rcm_comp_sizes<<<g3_grid_for(n_plus, 256), 256, 0, s>>>(B.p, n_plus, lo,
                                                            (unsigned long long*)B.base);
    G3_CHECK_LAUNCH();
  }
  G3_TRY(g3_exclusive_scan_i64(B.base, B.base, n_plus, s));
  G3_TRY(g3_alloc(&B.pos, n, s));
  G3_TRY(g3_alloc(&B.ppos, n, s));
  G3_TRY(g3_alloc(&B.front, (size_t)n_plus + 1, s));
  G3_TRY(g3_alloc(&B.next, (size_t)n_plus + 1, s));
  G3_TRY(g3_alloc(&B.fseg, (size_t)n_plus + 1, s));
  G3_TRY_CUDA(cudaMemsetAsync(B.pos, 0xFF, (size_t)n * sizeof(int32_t), s));
  G3_TRY_CUDA(cudaMemsetAsync(B.ppos, 0xFF, (size_t)n * sizeof(uint32_t), s));
  G3_TRY(g3_compact((int64_t)n_plus, IsRoot{B.p, lo},
                    EmitStart{B.vplus, B.base, B.pos, B.cursor, B.front}, B.partial, s));
  int64_t nf = 0;
  G3_TRY(read_i64(B.partial + (n_plus + CP_TILE - 1) / CP_TILE, &nf, s));

  // 4. Cuthill-McKee levels, all components at once
  const int bits_r = g3_bits_for(n_plus);
  while (nf > 0) {
    rcm_front_degrees<<<g3_grid_for(nf, 256), 256, 0, s>>>(B.front, nf, g->off, B.fseg);
    G3_CHECK_LAUNCH();
    G3_TRY(g3_exclusive_scan_i64(B.fseg, B.fseg, nf, s));
    G3_TRY_CUDA(cudaMemsetAsync(B.counters + 1, 0, sizeof(unsigned long long), s));
    rcm_expand<<<grid, 256, 0, s>>>(
        B.fseg, nf,
        ExpandLevel{B.front, B.fseg, g->off, g->col, B.pos, B.ppos, B.next, B.counters + 1,
                    B.rank, lo});
    G3_CHECK_LAUNCH();
    int64_t len = 0;
    G3_TRY(read_i64((const int64_t*)(B.counters + 1), &len, s));
    if (len == 0) break;
    rcm_level_keys<<<g3_grid_for(len, 256), 256, 0, s>>>(B.next, len, B.ppos, B.rank, bits_r,
                                                         B.ka);
    G3_CHECK_LAUNCH();
    G3_TRY(g3_radix_sort_u64(B.ka, B.kb, len, 2 * bits_r, &sorted, s));
    rcm_level_heads<<<g3_grid_for(len, 256), 256, 0, s>>>(sorted, len, bits_r, B.p, B.first);
    G3_CHECK_LAUNCH();
    rcm_level_place<<<g3_grid_for(len, 256), 256, 0, s>>>(sorted, len, bits_r, B.p, B.vplus,
                                                          B.first, B.cursor, B.pos, B.front);
    G3_CHECK_LAUNCH();
    rcm_level_tails<<<g3_grid_for(len, 256), 256, 0, s>>>(sorted, len, bits_r, B.p, B.first,
                                                          B.cursor);
    G3_CHECK_LAUNCH();
    nf = len;
  }

  // 5. labels, inverse, relabelled CSR
  rcm_labels<<<g3_grid_for(n, 256), 256, 0, s>>>(B.pos, n, k, g->new_of_old);
  G3_CHECK_LAUNCH();
  if (lo == 0 && n_plus > 0) {  // every component was ordered: keep their ranges
    G3_TRY(g3_alloc(&g->comp_rng, n_plus, s));
    rcm_comp_ranges<<<g3_grid_for(n, 256), 256, 0, s>>>(B.rank, B.p, B.base, B.cursor,
                                                        g->new_of_old, n, k, g->comp_rng);
    G3_CHECK_LAUNCH();
  }
  if (lo > 0)
    G3_TRY(g3_compact((int64_t)n, IsUnordered{g->off, B.rank, lo},
                      EmitUnorderedLabel{k, g->new_of_old}, B.partial, s));
  G3_TRY(g3_compact((int64_t)n, IsIsolated{g->off}, EmitIsolatedLabel{n_plus, g->new_of_old},
                    B.partial, s));
  G3_TRY(g3_alloc(&B.deg_new, (size_t)n_plus + 1, s));
  rcm_inverse<<<g3_grid_for(n, 256), 256, 0, s>>>(g->new_of_old, n, g->off, g->old_of_new,
                                                  B.deg_new);
  G3_CHECK_LAUNCH();
  int64_t* off_new;
  G3_TRY(g3_alloc(&off_new, (size_t)n_plus + 1, s));
  {
    const g3_status sc = g3_exclusive_scan_i64(B.deg_new, off_new, n_plus, s);
    if (sc != G3_OK) {
      g3_free(off_new, s);
      return sc;
    }
  }
  B.ka = (g3_free(B.ka, s), nullptr);
  B.kb = (g3_free(B.kb, s), nullptr);
  int32_t* col_new;
  g3_status st = g3_alloc(&col_new, nnz > 0 ? nnz : 1, s);
  if (st != G3_OK) {
    g3_free(off_new, s);
    return st;
  }
  if (nnz > 0) {
    const int bits_n = g3_bits_for(n_plus);
    st = g3_alloc(&B.ka, nnz, s);
    if (st == G3_OK) st = g3_alloc(&B.kb, nnz, s);
    if (st != G3_OK) {
      g3_free(off_new, s);
      g3_free(col_new, s);
      return st;
    }
    rcm_perm_keys<<<grid, 256, 0, s>>>(g->off, n, PermKey{g->col, g->new_of_old, B.ka, bits_n});
    g3_count_launch();
    st = cudaGetLastError() == cudaSuccess ? G3_OK : G3_ECUDA;
    if (st == G3_OK) st = g3_radix_sort_u64(B.ka, B.kb, nnz, 2 * bits_n, &sorted, s);
    if (st == G3_OK) {
      rcm_take_col<<<g3_grid_for(nnz, 256), 256, 0, s>>>(sorted, nnz, bits_n, col_new);
      g3_count_launch();
      if (cudaGetLastError() != cudaSuccess) st = G3_ECUDA;
    }
    if (st != G3_OK) {
      if (st == G3_ECUDA) g3_set_error("g3_rcm_relabel: relabelled CSR kernels failed");
      g3_free(off_new, s);
      g3_free(col_new, s);
      return st;
    }
  }
  g3_free(g->off, s);
  g3_free(g->col, s);
  g->off = off_new;
  g->col = col_new;
  g->n_bfs = n_plus;
  g->n_plus = n_plus;
  g->relabelled = 1;
  return G3_OK;
}

static g3_status relabel(g3_graph* g, int32_t p_permille, cudaStream_t s, const char* name) {
  if (!g) {
    g3_set_error("%s: graph is NULL", name);
    return G3_EINVAL;
  }
  if (p_permille < 0 || p_permille > 1000) {
    g3_set_error("%s: p_permille %d outside [0, 1000]", name, p_permille);
    return G3_EINVAL;
  }
  if (g->relabelled) {
    g3_set_error("%s: graph already relabelled", name);
    return G3_ESTATE;
  }
  if (g->ws || g->ms) {
    cudaStreamSynchronize(s);
    g3_bfs_ws_free(g->ws);
    g3_ms_ws_free(g->ms);
    g->ws = nullptr;
    g->ms = nullptr;
  }
  RcmBufs B;
  g3_status st = rcm_impl(g, p_permille, s, B);
  B.release(s);
  if (st == G3_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      g3_set_error("%s: %s", name, cudaGetErrorString(e));
      return G3_ECUDA;
    }
  } else {
    // the graph stays as it was (not relabelled, its CSR untouched); a
    // half-made permutation is dropped
    g3_free(g->new_of_old, s);
    g3_free(g->old_of_new, s);
    g3_free(g->comp_rng, s);
    g->new_of_old = g->old_of_new = nullptr;
    g->comp_rng = nullptr;
    cudaStreamSynchronize(s);
  }
  return st;
}

extern "C" g3_status g3_rcm_relabel(g3_graph* g, void* stream) {
  return relabel(g, 1000, (cudaStream_t)stream, "g3_rcm_relabel");
}

extern "C" g3_status g3_rcm_relabel_partial(g3_graph* g, int32_t p_permille, void* stream) {
  return relabel(g, p_permille, (cudaStream_t)stream, "g3_rcm_relabel_partial");
}
