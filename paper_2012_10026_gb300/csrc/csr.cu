// CSR construction (Sec. 3.1, Eq. 2): the undirected graph of the generated
// tuples, both directions stored, self-loops and duplicates removed, rows
// ascending. Each tuple (u, v) becomes the keys u<<b|v and v<<b|u (b = bits
// of n); one radix sort orders all keys by (row, neighbour); a stable
// compaction keeps the first of each run of equal keys; row lengths come from
// run boundaries and an exclusive scan gives the int64 row offsets.
#include <stdlib.h>

#include "g3_prims.cuh"

#define G3_SENTINEL 0xFFFFFFFFFFFFFFFFull

__global__ void csr_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                              int64_t m, int32_t n, int bits, uint64_t* __restrict__ keys,
                              int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[i], v = dst[i];
    ulonglong2 kv;
    if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
      *err = 1;
      kv.x = kv.y = G3_SENTINEL;
    } else if (u == v) {
      kv.x = kv.y = G3_SENTINEL;  // self-loop dropped
    } else {
      kv.x = ((uint64_t)u << bits) | (uint64_t)v;
      kv.y = ((uint64_t)v << bits) | (uint64_t)u;
    }
    reinterpret_cast<ulonglong2*>(keys)[i] = kv;
  }
}

struct KeepFirstOfRun {
  const uint64_t* k;
  __device__ bool operator()(int64_t i) const {
    uint64_t x = k[i];
    return x != G3_SENTINEL && (i == 0 || k[i - 1] != x);
  }
};
struct CopyKey {
  const uint64_t* in;
  uint64_t* out;
  __device__ void operator()(int64_t i, int64_t pos) const { out[pos] = in[i]; }
};

// deg[u] receives (last + 1) - first over the run of row u.
__global__ void csr_rows(const uint64_t* __restrict__ ck, int64_t nnz, int bits,
                         int32_t* __restrict__ col, unsigned long long* deg) {
  const uint64_t mask = (1ull << bits) - 1ull;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = ck[p];
    uint64_t u = key >> bits;
    col[p] = (int32_t)(key & mask);
    if (p == 0 || (ck[p - 1] >> bits) != u) atomicAdd(&deg[u], (unsigned long long)(-p));
    if (p == nnz - 1 || (ck[p + 1] >> bits) != u) atomicAdd(&deg[u], (unsigned long long)(p + 1));
  }
}

__global__ void csr_max_degree(const int64_t* __restrict__ off, int32_t n,
                               unsigned long long* out) {
  unsigned long long mx = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
    mx = d > mx ? d : mx;
  }
  for (int o = 16; o; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

g3_status g3_graph_max_degree(g3_graph* g, cudaStream_t s) {
  unsigned long long* d;
  G3_TRY(g3_alloc(&d, 1, s));
  unsigned long long h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), s);
  if (e == cudaSuccess && g->n_bfs > 0) {
    csr_max_degree<<<g3_grid_for(g->n_bfs, 256), 256, 0, s>>>(g->off, g->n_bfs, d);
    g3_count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  g3_free(d, s);
  if (e != cudaSuccess) {
    g3_set_error("g3_graph_max_degree: %s", cudaGetErrorString(e));
    return G3_ECUDA;
  }
  g->max_degree = (int64_t)h;
  return G3_OK;
}

// Temporaries of the build, released on every path (a failure part-way
// leaves nothing allocated but what the graph itself owns, which
// g3_build_csr frees with the graph).
struct BuildBufs {
  uint64_t *ka = nullptr, *kb = nullptr;
  int64_t* partial = nullptr;
  int* err = nullptr;
  unsigned long long* deg = nullptr;
  void release(cudaStream_t s) {
    void* all[] = {ka, kb, partial, err, deg};
    for (void* x : all) g3_free(x, s);
  }
};

static g3_status build_impl(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                            cudaStream_t s, g3_graph* g, BuildBufs& B) {
  const int bits = g3_bits_for(n);
  const int64_t nk = 2 * m;
  uint64_t* sorted = nullptr;
  int64_t host[2] = {0, 0};

  g->n = n;
  g->n_bfs = n;
  G3_TRY(g3_alloc(&g->off, (size_t)n + 1, s));
  if (nk == 0) {
    G3_TRY_CUDA(cudaMemsetAsync(g->off, 0, ((size_t)n + 1) * sizeof(int64_t), s));
    G3_TRY(g3_alloc(&g->col, 1, s));
    g->nnz = 0;
    return g3_graph_max_degree(g, s);
  }
  G3_TRY(g3_alloc(&B.ka, nk, s));
  G3_TRY(g3_alloc(&B.kb, nk, s));
  G3_TRY(g3_alloc(&B.err, 2, s));
  G3_TRY_CUDA(cudaMemsetAsync(B.err, 0, sizeof(int), s));
  csr_make_keys<<<g3_grid_for(m, 256), 256, 0, s>>>(src, dst, m, n, bits, B.ka, B.err);
  G3_CHECK_LAUNCH();
  G3_TRY(g3_radix_sort_u64(B.ka, B.kb, nk, 2 * bits, &sorted, s));
  uint64_t* other = sorted == B.ka ? B.kb : B.ka;
  G3_TRY(g3_alloc(&B.partial, g3_compact_partials(nk), s));
  G3_TRY(g3_compact(nk, KeepFirstOfRun{sorted}, CopyKey{sorted, other}, B.partial, s));
  int64_t nbk = (nk + CP_TILE - 1) / CP_TILE;
  G3_TRY_CUDA(cudaMemcpyAsync(&host[0], B.partial + nbk, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, s));
  int herr = 0;
  G3_TRY_CUDA(cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    g3_set_error("g3_build_csr: an endpoint lies outside [0, %d)", n);
    return G3_EINVAL;
  }
  const int64_t nnz = host[0];
  g->nnz = nnz;
  G3_TRY(g3_alloc(&g->col, nnz > 0 ? nnz : 1, s));
  G3_TRY(g3_alloc(&B.deg, (size_t)n + 1, s));
  G3_TRY_CUDA(cudaMemsetAsync(B.deg, 0, ((size_t)n + 1) * sizeof(*B.deg), s));
  if (nnz > 0) {
    csr_rows<<<g3_grid_for(nnz, 256), 256, 0, s>>>(other, nnz, bits, g->col, B.deg);
    G3_CHECK_LAUNCH();
  }
  G3_TRY(g3_exclusive_scan_i64((const int64_t*)B.deg, g->off, n, s));
  B.release(s);
  B = BuildBufs();
  return g3_graph_max_degree(g, s);
}

extern "C" g3_status g3_build_csr(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                                  void* stream, g3_graph** out) {
  if (!out) {
    g3_set_error("g3_build_csr: out is NULL");
    return G3_EINVAL;
  }
  *out = nullptr;
  if (n <= 0 || m < 0 || m > (1ll << 40) || (m > 0 && (!src || !dst))) {
    g3_set_error("g3_build_csr: bad arguments (n=%d, m=%lld)", n, (long long)m);
    return G3_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  g3_graph* g = (g3_graph*)calloc(1, sizeof(g3_graph));
  if (!g) return G3_ENOMEM;
  BuildBufs B;
  g3_status st = build_impl(src, dst, m, n, s, g, B);
  B.release(s);
  if (st != G3_OK) {
    cudaStreamSynchronize(s);
    g3_graph_free(g);
    return st;
  }
  *out = g;
  return G3_OK;
}
