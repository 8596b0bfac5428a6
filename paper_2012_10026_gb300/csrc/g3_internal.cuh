// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "g3bfs.h"

#define G3_BLOCK 256
#define G3_NUM_SMS 152

// ----------------------------------------------------------------- errors
void g3_set_error(const char* fmt, ...);

#define G3_TRY_CUDA(expr)                                                   \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) {                                                \
      g3_set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,              \
                   cudaGetErrorString(_e));                                 \
      return _e == cudaErrorMemoryAllocation ? G3_ENOMEM : G3_ECUDA;        \
    }                                                                       \
  } while (0)

#define G3_TRY(expr)                  \
  do {                                \
    g3_status _s = (expr);            \
    if (_s != G3_OK) return _s;       \
  } while (0)

// Every kernel launch site is followed by G3_CHECK_LAUNCH(), which also
// counts the launch (g3_kernel_launches()).
void g3_count_launch();
#define G3_CHECK_LAUNCH()                    \
  do {                                       \
    g3_count_launch();                       \
    G3_TRY_CUDA(cudaGetLastError());         \
  } while (0)

// ------------------------------------------------------------ allocation
// Stream-ordered device allocation that reports G3_ENOMEM.
g3_status g3_malloc(void** p, size_t bytes, cudaStream_t s);
void g3_free(void* p, cudaStream_t s);
// Fault-injection test hooks (g3_debug_inject): every device allocation
// site asks g3_alloc_should_fail() first and reports G3_ENOMEM when told to.
bool g3_alloc_should_fail();
int g3_rcm_hook_cap();
g3_status g3_bfs_set_staged_stall(int spins);

template <typename T>
static inline g3_status g3_alloc(T** p, size_t count, cudaStream_t s) {
  return g3_malloc((void**)p, count * sizeof(T) + 16, s);
}

// ------------------------------------------------------------ primitives
static inline int g3_bits_for(int64_t n) {  // bits to hold values < n (>= 1)
  int b = 1;
  while ((1LL << b) < n) ++b;
  return b;
}
static inline int g3_grid_for(int64_t items, int per_block, int cap = G3_NUM_SMS * 16) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

// Radix sort of n uint64 keys by their low `nbits` bits, ascending and
// stable. `keys` and `tmp` hold n entries each; the sorted keys end in
// *result (== keys or tmp).
g3_status g3_radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int nbits,
                            uint64_t** result, cudaStream_t s);

// Exclusive prefix sum of n int64 values into out (n+1 entries: out[n] is the
// total). in and out may alias.
g3_status g3_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- graph
struct g3_bfs_ws;  // BFS workspace (bfs.cu)
struct g3_ms_ws;   // multi-source BFS workspace (msbfs.cu)

struct g3_graph {
  int32_t n;            // vertices of the input
  int64_t nnz;          // directed entries
  int64_t max_degree;
  int32_t n_bfs;        // rows of the current CSR (n or n_plus)
  int32_t n_plus;
  int relabelled;
  int64_t* off;         // current CSR [n_bfs + 1]
  int32_t* col;         // [nnz]
  int32_t* old_of_new;  // [n] after relabel
  int32_t* new_of_old;  // [n] after relabel
  // [n_plus] after a full RCM relabel, else NULL: the label range [x, y) of
  // each label's connected component (Algorithm 3 numbers a component's
  // vertices consecutively, so every component is one range of labels)
  int2* comp_rng;
  g3_bfs_ws* ws;
  g3_ms_ws* ms;
};

void g3_bfs_ws_free(g3_bfs_ws* ws);
// Search from several roots at once (device array; root i counts when it lies
// in [lo[i], lo[i+1]), lo nullable); used by the batched search over a union
// of disjoint graphs. Synchronises.
g3_status g3_bfs_multi_root(g3_graph* g, const int32_t* roots, int32_t count, const int32_t* lo,
                            const g3_bfs_opts* opts, int32_t* parent, int32_t* level,
                            cudaStream_t s);
void g3_ms_ws_free(g3_ms_ws* ws);

// ----------------------------------------------------------- device utils
__device__ __forceinline__ unsigned g3_lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ int g3_lane() { return threadIdx.x & 31; }

// Warp-aggregated append of `item` (when `want`) to queue/len. Every lane in
// `mask` must call it with the same mask.
__device__ __forceinline__ void g3_warp_append(unsigned mask, bool want, int32_t item,
                                               int32_t* queue, unsigned long long* len) {
  unsigned bal = __ballot_sync(mask, want);
  if (bal == 0) return;
  int leader = __ffs(bal) - 1;
  unsigned long long base = 0;
  if (g3_lane() == leader) base = atomicAdd(len, (unsigned long long)__popc(bal));
  base = __shfl_sync(mask, base, leader);
  if (want) queue[base + __popc(bal & g3_lanemask_lt())] = item;
}
