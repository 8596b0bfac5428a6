// Device-wide building blocks used by the CSR builder and the RCM relabeller:
// stable compaction (select) with a caller functor, and block-level helpers.
#pragma once
#include "g3_internal.cuh"

#define CP_THREADS 256
#define CP_IPT 16
#define CP_TILE (CP_THREADS * CP_IPT)  // 4096 items per block

// Exclusive scan of nb int64 partials in place (single block). Defined in
// sort.cu.
g3_status g3_scan_partials(int64_t* partial, int64_t nb, cudaStream_t s);

// Block-wide exclusive scan of one value per thread (blockDim.x == 256).
// Returns the exclusive prefix; *total receives the block sum.
__device__ __forceinline__ int64_t g3_block_excl_scan_256(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  int64_t woff = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    int64_t x = wsum[w];
    if (w < warp) woff += x;
    tot += x;
  }
  __syncthreads();
  *total = tot;
  return woff + inc - v;
}

// Pass 1: per-tile count of items i in [0, n) with pred(i).
template <class Pred>
__global__ void __launch_bounds__(CP_THREADS) g3_compact_count(int64_t n, Pred pred,
                                                               int64_t* partial) {
  const int64_t base = (int64_t)blockIdx.x * CP_TILE;
  int64_t c = 0;
#pragma unroll 4
  for (int k = 0; k < CP_IPT; ++k) {
    int64_t i = base + (int64_t)k * CP_THREADS + threadIdx.x;
    if (i < n && pred(i)) ++c;
  }
  int64_t tot;
  g3_block_excl_scan_256(c, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Pass 2: emit(i, position) for every selected i, positions in index order.
template <class Pred, class Emit>
__global__ void __launch_bounds__(CP_THREADS) g3_compact_scatter(int64_t n, Pred pred,
                                                                 Emit emit,
                                                                 const int64_t* partial) {
  __shared__ unsigned cnt[CP_IPT][8];
  __shared__ int64_t off[CP_IPT][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * CP_TILE;
  unsigned bal[CP_IPT];
#pragma unroll
  for (int k = 0; k < CP_IPT; ++k) {
    int64_t i = base + (int64_t)k * CP_THREADS + threadIdx.x;
    bool p = i < n && pred(i);
    bal[k] = __ballot_sync(0xffffffffu, p);
    if (lane == 0) cnt[k][warp] = __popc(bal[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = partial[blockIdx.x];
    for (int k = 0; k < CP_IPT; ++k)
      for (int w = 0; w < 8; ++w) {
        off[k][w] = run;
        run += cnt[k][w];
      }
  }
  __syncthreads();
  const unsigned lt = g3_lanemask_lt();
#pragma unroll
  for (int k = 0; k < CP_IPT; ++k) {
    if (bal[k] & (1u << lane)) {
      int64_t i = base + (int64_t)k * CP_THREADS + threadIdx.x;
      emit(i, off[k][warp] + __popc(bal[k] & lt));
    }
  }
}

// Stable compaction over [0, n): emit(i, pos) for each i with pred(i), pos
// counting the selected items in index order. partial must hold
// ceil(n / CP_TILE) + 1 int64 entries; *d_total (device) gets the count.
template <class Pred, class Emit>
g3_status g3_compact(int64_t n, Pred pred, Emit emit, int64_t* partial, cudaStream_t s) {
  int64_t nb = (n + CP_TILE - 1) / CP_TILE;
  if (nb == 0) {
    G3_TRY_CUDA(cudaMemsetAsync(partial, 0, sizeof(int64_t), s));
    return G3_OK;
  }
  g3_compact_count<Pred><<<(unsigned)nb, CP_THREADS, 0, s>>>(n, pred, partial);
  G3_CHECK_LAUNCH();
  G3_TRY(g3_scan_partials(partial, nb, s));  // partial[nb] = total
  g3_compact_scatter<Pred, Emit><<<(unsigned)nb, CP_THREADS, 0, s>>>(n, pred, emit, partial);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

static inline int64_t g3_compact_partials(int64_t n) { return (n + CP_TILE - 1) / CP_TILE + 1; }

// First index i in [0, n) with a[i] > x (a ascending); n when none.
__device__ __forceinline__ int64_t g3_upper_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Edge-parallel walk over a CSR-like segment structure with `rows` rows and
// row offsets seg[0..rows] (ascending, seg[0] = 0): every warp of the grid
// owns an equal contiguous range of entries, lanes take consecutive entries
// (coalesced), and each lane tracks the row its entry belongs to. Calls
// f(row, entry, active) with the whole warp converged; only calls with
// active == true carry an entry of [0, seg[rows]). Balanced whatever the
// degree skew (the GPU form of splitting long lists evenly, Algorithm 4).
template <class F>
__device__ __forceinline__ void g3_for_each_entry(const int64_t* seg, int64_t rows, F& f) {
  const int64_t total = seg[rows];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t per = (((total + nwarps - 1) / nwarps) + 31) & ~31ll;
  const int64_t j0 = warp * per, j1 = min(total, j0 + per);
  if (j0 >= j1) return;  // warp-uniform
  int64_t r = g3_upper_bound_i64(seg, rows + 1, j0) - 1;  // row holding j0
  for (int64_t base = j0; base < j1; base += 32) {
    const int64_t j = base + lane;
    const bool active = j < j1;
    if (active) {
      while (seg[r + 1] <= j) ++r;
    }
    f(r, j, active);
  }
}
