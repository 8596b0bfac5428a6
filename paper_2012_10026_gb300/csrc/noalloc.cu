// g3_bfs_noalloc: a top-down BFS entry point that allocates no memory.
//
// Who needs it: callers that cannot call cudaMalloc / cudaFree (or anything
// that allocates) at the point where they run a search -- for example code
// living inside a host framework that has already reserved the device memory
// for its own pool, or latency-critical paths where an allocation or free
// could synchronise the device. g3_bfs allocates its workspace on the first
// call for each graph; this variant instead keeps its scratch (visited bitmap,
// two frontier queues, two counters) in one file-scope __device__ array of
// fixed size, and the caller passes the CSR and the outputs.
//
// Limits and sharing:
//   * at most G3_NOALLOC_MAX_N vertices; larger graphs are rejected with
//     G3_EINVAL before anything runs. The array takes 8,519,936 bytes (about
//     8.5 MB) of device memory on every GPU that loads the library, until
//     the process exits.
//   * every call on a device uses the same array, and the array keeps the
//     last call's contents; each call clears the parts that must start at
//     zero. Calls whose GPU work overlaps (other streams, other host threads)
//     race on the array: serialise them.
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it for the
//     life of the process; make that first call before any stream capture.
//     The cached address belongs to the device's context at that time: after
//     cudaDeviceReset on that device, do not call this entry point again.
#include <mutex>

#include "g3_internal.cuh"

#define NA_MAX_N (1 << 20)
#define NA_WORDS (NA_MAX_N / 32)
// layout: [visited: NA_WORDS u32][queue 0: NA_MAX_N i32][queue 1: NA_MAX_N i32]
//         [counters: 4 u64]
#define NA_OFF_Q0 ((size_t)NA_WORDS * 4)
#define NA_OFF_Q1 (NA_OFF_Q0 + (size_t)NA_MAX_N * 4)
#define NA_OFF_CTR (NA_OFF_Q1 + (size_t)NA_MAX_N * 4)
#define NA_BYTES (NA_OFF_CTR + 256)

static __device__ __align__(256) unsigned char g3_noalloc_scratch[NA_BYTES];

#define NA_MAX_DEVICES 64
static std::mutex na_mutex;
static unsigned char* na_scratch_addr[NA_MAX_DEVICES];

// Device address of the scratch array on the current device (looked up once
// per device).
static g3_status na_scratch(unsigned char** out) {
  int dev = 0;
  G3_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) {
    g3_set_error("g3_bfs_noalloc: device ordinal %d beyond %d", dev, NA_MAX_DEVICES);
    return G3_EINVAL;
  }
  std::lock_guard<std::mutex> lock(na_mutex);
  if (!na_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g3_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      g3_set_error("g3_bfs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return G3_ECUDA;
    }
    na_scratch_addr[dev] = (unsigned char*)p;
  }
  *out = na_scratch_addr[dev];
  return G3_OK;
}

__global__ void na_init(int32_t n, uint32_t* visited, int32_t* parent, int32_t* level,
                        unsigned long long* ctr) {
  const int64_t words = ((int64_t)n + 31) / 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    parent[i] = -1;
    level[i] = -1;
    if (i < words) visited[i] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) ctr[threadIdx.x] = 0ull;
}

__global__ void na_root(int32_t root, uint32_t* visited, int32_t* parent, int32_t* level,
                        int32_t* q0, unsigned long long* ctr) {
  visited[root >> 5] |= 1u << (root & 31);
  parent[root] = root;
  level[root] = 0;
  q0[0] = root;
  ctr[0] = 1ull;
}

// One warp per frontier vertex; lanes stride over its neighbour list. A
// neighbour is claimed by atomicOr on its visited word; the winner writes
// parent/level and appends it to the next queue (one atomic per warp step).
__global__ void __launch_bounds__(256) na_expand(const int64_t* __restrict__ off,
                                                 const int32_t* __restrict__ col,
                                                 const int32_t* __restrict__ q,
                                                 const unsigned long long* cur_len,
                                                 int32_t* qn, unsigned long long* next_len,
                                                 uint32_t* visited, int32_t* parent,
                                                 int32_t* level, int32_t lnext) {
  const int64_t len = (int64_t)*cur_len;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < len; i += nwarps) {
    const int32_t v = q[i];
    const int64_t b = off[v], e = off[v + 1];
    for (int64_t base = b; base < e; base += 32) {
      const int64_t j = base + lane;
      bool claim = false;
      int32_t w = 0;
      if (j < e) {
        w = col[j];
        const uint32_t bit = 1u << (w & 31);
        if (!(__ldcg(&visited[w >> 5]) & bit)) claim = !(atomicOr(&visited[w >> 5], bit) & bit);
        if (claim) {
          parent[w] = v;
          level[w] = lnext;
        }
      }
      g3_warp_append(0xffffffffu, claim, w, qn, next_len);
    }
  }
}

extern "C" g3_status g3_bfs_noalloc(const int64_t* off, const int32_t* col, int32_t n,
                                    int32_t root, int32_t* parent, int32_t* level,
                                    void* stream) {
  if (n <= 0 || n > NA_MAX_N) {
    g3_set_error("g3_bfs_noalloc: n = %d outside [1, %d] (the static scratch holds at most "
                 "%d vertices)", n, NA_MAX_N, NA_MAX_N);
    return G3_EINVAL;
  }
  if (!off || !col || !parent || !level) {
    g3_set_error("g3_bfs_noalloc: null pointer argument");
    return G3_EINVAL;
  }
  if (root < 0 || root >= n) {
    g3_set_error("g3_bfs_noalloc: root %d outside [0, %d)", root, n);
    return G3_EINVAL;
  }
  unsigned char* base = nullptr;
  G3_TRY(na_scratch(&base));
  uint32_t* visited = (uint32_t*)base;
  int32_t* q[2] = {(int32_t*)(base + NA_OFF_Q0), (int32_t*)(base + NA_OFF_Q1)};
  unsigned long long* ctr = (unsigned long long*)(base + NA_OFF_CTR);
  cudaStream_t s = (cudaStream_t)stream;

  na_init<<<g3_grid_for(n, 256), 256, 0, s>>>(n, visited, parent, level, ctr);
  G3_CHECK_LAUNCH();
  na_root<<<1, 1, 0, s>>>(root, visited, parent, level, q[0], ctr);
  G3_CHECK_LAUNCH();
  int cur = 0;
  for (int32_t L = 0;; ++L) {
    unsigned long long len = 0;
    G3_TRY_CUDA(cudaMemcpyAsync(&len, ctr + cur, sizeof(len), cudaMemcpyDeviceToHost, s));
    G3_TRY_CUDA(cudaStreamSynchronize(s));
    if (len == 0) break;
    G3_TRY_CUDA(cudaMemsetAsync(ctr + (1 - cur), 0, sizeof(unsigned long long), s));
    na_expand<<<g3_grid_for((int64_t)len, 8, G3_NUM_SMS * 16), 256, 0, s>>>(
        off, col, q[cur], ctr + cur, q[1 - cur], ctr + (1 - cur), visited, parent, level,
        L + 1);
    G3_CHECK_LAUNCH();
    cur = 1 - cur;
  }
  return G3_OK;
}
