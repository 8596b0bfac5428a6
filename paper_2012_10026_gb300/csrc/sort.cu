// Device-wide primitives: LSD radix sort of uint64 keys, exclusive scans,
// stream-ordered allocation and the error-detail buffer.
#include <stdarg.h>
#include <string.h>

#include <atomic>

#include "g3_prims.cuh"

// ---------------------------------------------------------------- errors
static thread_local char g_err[512];

void g3_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* g3_last_error_detail(void) { return g_err; }

extern "C" const char* g3_status_str(g3_status s) {
  switch (s) {
    case G3_OK: return "ok";
    case G3_EINVAL: return "invalid argument";
    case G3_ENOMEM: return "out of memory";
    case G3_ECUDA: return "CUDA error";
    case G3_ETIMEOUT: return "device-side wait timed out";
    case G3_ERANGE: return "result out of range for the output type";
    case G3_ESTATE: return "call not valid in the current state";
  }
  return "unknown status";
}

extern "C" const char* g3_version(void) { return "g3bfs 0.1 sm_103a"; }

static std::atomic<unsigned long long> g_launches{0};
void g3_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" uint64_t g3_kernel_launches(void) { return g_launches.load(); }

// ---------------------------------------------------- fault injection
// Test hooks (g3_debug_inject): fail the k-th device allocation after arming
// (one shot), and cap the component-hooking rounds of the RCM relabel.
static std::atomic<long long> g_fail_at{0};
static std::atomic<long long> g_alloc_seen{0};
static std::atomic<int> g_hook_cap{4096};

bool g3_alloc_should_fail() {
  if (g_fail_at.load(std::memory_order_relaxed) <= 0) return false;
  const long long c = g_alloc_seen.fetch_add(1) + 1;
  long long k = c;
  if (g_fail_at.compare_exchange_strong(k, 0)) {
    g3_set_error("device allocation %lld failed (injected)", c);
    return true;
  }
  return false;
}

int g3_rcm_hook_cap() { return g_hook_cap.load(std::memory_order_relaxed); }

extern "C" g3_status g3_debug_inject(int32_t kind, int64_t value) {
  if (kind == G3_INJECT_ALLOC) {
    g_alloc_seen = 0;
    g_fail_at = value > 0 ? value : 0;
    return G3_OK;
  }
  if (kind == G3_INJECT_STAGED_STALL) return g3_bfs_set_staged_stall(value > 0 ? (int)value : 0);
  if (kind == G3_INJECT_RCM_ROUNDS) {
    g_hook_cap = value > 0 ? (int)(value < (1 << 30) ? value : (1 << 30)) : 4096;
    return G3_OK;
  }
  g3_set_error("g3_debug_inject: unknown kind %d", kind);
  return G3_EINVAL;
}

extern "C" g3_status g3_debug_pool_used(int64_t* bytes) {
  if (!bytes) {
    g3_set_error("g3_debug_pool_used: null argument");
    return G3_EINVAL;
  }
  int dev = 0;
  cudaMemPool_t pool;
  G3_TRY_CUDA(cudaGetDevice(&dev));
  G3_TRY_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t used = 0;
  G3_TRY_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *bytes = (int64_t)used;
  return G3_OK;
}

g3_status g3_malloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (g3_alloc_should_fail()) return G3_ENOMEM;
  cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    g3_set_error("cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? G3_ENOMEM : G3_ECUDA;
  }
  return G3_OK;
}

void g3_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// ------------------------------------------------------------------ scans
// Single-block exclusive scan of nb int64 values in place; partial[nb] gets
// the total. Each of the 1024 threads owns one contiguous segment.
__global__ void __launch_bounds__(1024) g3_scan_partials_kernel(int64_t* p, int64_t nb) {
  __shared__ int64_t seg[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b = t * per, e = min(nb, b + per);
  int64_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += p[i];
  seg[t] = sum;
  __syncthreads();
  // Hillis-Steele over 1024 segment sums
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t x = t >= o ? seg[t - o] : 0;
    __syncthreads();
    seg[t] += x;
    __syncthreads();
  }
  int64_t run = seg[t] - sum;  // exclusive
  for (int64_t i = b; i < e; ++i) {
    int64_t x = p[i];
    p[i] = run;
    run += x;
  }
  if (t == 1023) p[nb] = seg[1023];
}

g3_status g3_scan_partials(int64_t* partial, int64_t nb, cudaStream_t s) {
  g3_scan_partials_kernel<<<1, 1024, 0, s>>>(partial, nb);
  G3_CHECK_LAUNCH();
  return G3_OK;
}

#define SC_TILE 4096  // 256 threads x 16 items

__global__ void __launch_bounds__(256) g3_scan_reduce(const int64_t* in, int64_t n,
                                                      int64_t* partial) {
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
  int64_t c = 0;
  for (int k = 0; k < 16; ++k) {
    int64_t i = base + k * 256 + threadIdx.x;
    if (i < n) c += in[i];
  }
  int64_t tot;
  g3_block_excl_scan_256(c, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) g3_scan_down(const int64_t* in, int64_t* out, int64_t n,
                                                    const int64_t* partial, int64_t nb) {
  __shared__ int64_t tile[SC_TILE];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
  for (int k = 0; k < 16; ++k) {
    int64_t i = base + k * 256 + threadIdx.x;
    tile[k * 256 + threadIdx.x] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int64_t v[16], c = 0;
  for (int k = 0; k < 16; ++k) {
    v[k] = tile[threadIdx.x * 16 + k];
    c += v[k];
  }
  int64_t tot;
  int64_t run = g3_block_excl_scan_256(c, &tot) + partial[blockIdx.x];
  for (int k = 0; k < 16; ++k) {
    tile[threadIdx.x * 16 + k] = run;
    run += v[k];
  }
  __syncthreads();
  for (int k = 0; k < 16; ++k) {
    int64_t i = base + k * 256 + threadIdx.x;
    if (i < n) out[i] = tile[k * 256 + threadIdx.x];
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = partial[nb];
}

g3_status g3_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  int64_t nb = (n + SC_TILE - 1) / SC_TILE;
  if (nb == 0) {
    G3_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return G3_OK;
  }
  int64_t* partial;
  G3_TRY(g3_alloc(&partial, nb + 1, s));
  g3_scan_reduce<<<(unsigned)nb, 256, 0, s>>>(in, n, partial);
  G3_CHECK_LAUNCH();
  G3_TRY(g3_scan_partials(partial, nb, s));
  g3_scan_down<<<(unsigned)nb, 256, 0, s>>>(in, out, n, partial, nb);
  G3_CHECK_LAUNCH();
  g3_free(partial, s);
  return G3_OK;
}

// ------------------------------------------------------------ radix sort
// LSD radix sort, 8-bit digits. Each of nb blocks owns a contiguous chunk of
// the keys (a multiple of RS_TILE). Per pass: (1) per-block digit histogram,
// (2) digit-major exclusive scan of the nb x 256 counts, (3) per-block stable
// scatter: each 2048-key tile is ranked in shared memory (warp match on the
// digit, then offsets across warps and digits), staged so that each digit's
// run is written out contiguously.
#define RS_THREADS 256
#define RS_WARPS 8
#define RS_KPT 8
#define RS_TILE (RS_THREADS * RS_KPT)

__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint64_t* __restrict__ keys,
                                                         int64_t n, int64_t chunk, int shift,
                                                         int64_t* hist, int nb) {
  __shared__ unsigned h[RS_WARPS][256];
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t begin = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(n, begin + chunk);
  const int warp = threadIdx.x >> 5;
  for (int64_t i = begin + threadIdx.x; i < end; i += RS_THREADS)
    atomicAdd(&h[warp][(unsigned)(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    int64_t c = 0;
    for (int w = 0; w < RS_WARPS; ++w) c += h[w][d];
    hist[(int64_t)d * nb + blockIdx.x] = c;
  }
}

__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint64_t* __restrict__ in,
                                                           uint64_t* __restrict__ out,
                                                           int64_t n, int64_t chunk, int shift,
                                                           const int64_t* __restrict__ hist,
                                                           int nb) {
  __shared__ int64_t run[256];
  __shared__ unsigned wcnt[RS_WARPS][256];
  __shared__ unsigned tile_excl[256];
  __shared__ unsigned tile_tot[256];
  __shared__ uint64_t stage[RS_TILE];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned lt = g3_lanemask_lt();
  run[tid] = hist[(int64_t)tid * nb + blockIdx.x];
  const int64_t begin = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(n, begin + chunk);
  for (int64_t tile = begin; tile < end; tile += RS_TILE) {
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    uint64_t k[RS_KPT];
    unsigned dig[RS_KPT], rank[RS_KPT];
    const int64_t wbase = tile + (int64_t)warp * (32 * RS_KPT);
#pragma unroll
    for (int j = 0; j < RS_KPT; ++j) {
      int64_t idx = wbase + j * 32 + lane;
      bool valid = idx < end;
      uint64_t key = valid ? in[idx] : 0ull;
      unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
      unsigned peers = __match_any_sync(0xffffffffu, d);
      unsigned before = __popc(peers & lt);
      unsigned base = d < 256u ? wcnt[warp][d] : 0u;
      __syncwarp();
      if (d < 256u && before == 0) wcnt[warp][d] = base + __popc(peers);
      __syncwarp();
      k[j] = key;
      dig[j] = d;
      rank[j] = base + before;
    }
    __syncthreads();
    {  // per digit: offsets of each warp's keys inside the digit's tile run
      unsigned r = 0;
      for (int w = 0; w < RS_WARPS; ++w) {
        unsigned c = wcnt[w][tid];
        wcnt[w][tid] = r;
        r += c;
      }
      tile_tot[tid] = r;
    }
    int64_t tot;
    int64_t ex = g3_block_excl_scan_256((int64_t)tile_tot[tid], &tot);
    tile_excl[tid] = (unsigned)ex;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_KPT; ++j) {
      if (dig[j] < 256u) stage[tile_excl[dig[j]] + wcnt[warp][dig[j]] + rank[j]] = k[j];
    }
    __syncthreads();
    const int cnt = (int)tot;
    for (int i = tid; i < cnt; i += RS_THREADS) {
      uint64_t key = stage[i];
      unsigned d = (unsigned)(key >> shift) & 255u;
      out[run[d] + (i - (int)tile_excl[d])] = key;
    }
    __syncthreads();
    run[tid] += tile_tot[tid];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) rs_scan_hist(int64_t* hist, int64_t total) {
  // exclusive scan in place (digit-major), one block
  __shared__ int64_t seg[1024];
  const int t = threadIdx.x;
  const int64_t per = (total + 1023) / 1024;
  const int64_t b = t * per, e = min(total, b + per);
  int64_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += hist[i];
  seg[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t x = t >= o ? seg[t - o] : 0;
    __syncthreads();
    seg[t] += x;
    __syncthreads();
  }
  int64_t r = seg[t] - sum;
  for (int64_t i = b; i < e; ++i) {
    int64_t x = hist[i];
    hist[i] = r;
    r += x;
  }
}

g3_status g3_radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int nbits,
                            uint64_t** result, cudaStream_t s) {
  *result = keys;
  if (n <= 1 || nbits <= 0) return G3_OK;
  int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
  int64_t nb = tiles < G3_NUM_SMS * 8 ? tiles : G3_NUM_SMS * 8;
  int64_t chunk = ((tiles + nb - 1) / nb) * RS_TILE;
  nb = (n + chunk - 1) / chunk;
  int64_t* hist;
  G3_TRY(g3_alloc(&hist, nb * 256, s));
  uint64_t *a = keys, *b = tmp;
  for (int shift = 0; shift < nbits; shift += 8) {
    rs_upsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(a, n, chunk, shift, hist, (int)nb);
    G3_CHECK_LAUNCH();
    rs_scan_hist<<<1, 1024, 0, s>>>(hist, nb * 256);
    G3_CHECK_LAUNCH();
    rs_downsweep<<<(unsigned)nb, RS_THREADS, 0, s>>>(a, b, n, chunk, shift, hist, (int)nb);
    G3_CHECK_LAUNCH();
    uint64_t* t = a;
    a = b;
    b = t;
  }
  g3_free(hist, s);
  *result = a;
  return G3_OK;
}
