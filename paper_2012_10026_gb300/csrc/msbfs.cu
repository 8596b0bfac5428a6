// Bit-sliced multi-source BFS: up to 64 searches at once, one bit per source
// in a uint64 per vertex (the paper's method has no multi-source form; this
// batches the roots of Sec. 4's 64-root evaluation into one pass).
//
// State per BFS-graph vertex v: vis[v] (sources that reached v), F[v] (sources
// whose frontier contains v). Level L -> L+1 runs one of two kernels:
//   push (small frontiers, the top-down analogue): every frontier vertex u
//     ORs F[u] & ~vis[w] into N[w] of each neighbour w; the first toucher of w
//     queues it; a finalize pass over the touched vertices keeps the new bits.
//   pull (large frontiers, the bottom-up analogue): every vertex not yet
//     reached by all sources ORs the frontier words of its neighbours, with an
//     early exit once every missing source is found; vertices with degree >=
//     pull_warp_deg are pulled by a whole warp (degree binning).
// Rows longer than MS_CHUNK entries (the hubs of a power-law graph) are split
// in both directions: the warp that meets such a row takes its first chunk
// and queues the others as (vertex, chunk) items for a follow-up kernel with
// one warp per item, so no single warp walks a million-entry row.
// Levels are stored per vertex as a 64-byte row in label order and written to
// level[s][original ID] (int8) by a shared-memory transpose at the end.
#include <string.h>

#include "g3_prims.cuh"

#define MS_CHUNK 2048  // row entries per warp work item

// Device counters (ctr[]): per level [0] next queue length, [1] next sum of
// degrees, [2] heavy / touched length, [3] chunk items, [4] pending heavy
// vertices; per call [5] row entries read and [6] vertices scanned by pull
// levels; the device-side level loop's state:
#define MS_QCUR 7     // length of the queue being expanded
#define MS_LEVEL 8    // levels expanded so far
#define MS_PULLS 9    // pull levels
#define MS_PUSHES 10  // push levels
#define MS_PUSHED 11  // row entries pushed
#define MS_ERANGE 12  // a level above 126 exists
#define MS_LNEXT 13   // the level the current expansion writes
#define MS_NCTR 32

struct g3_ms_ws {
  int32_t nb;
  uint64_t *vis, *fa, *fb, *nx;
  int8_t* lv;        // [nb][64]
  int32_t *qa, *qb;  // frontier queues
  int32_t* heavy;    // pull: vertices pulled by a warp
  int32_t* pend;     // pull: heavy vertices whose rows were split into chunks
  int2* items;       // (vertex, chunk index >= 1) of split rows
  int64_t items_cap;
  unsigned long long* ctr;  // MS_NCTR counters, see above
  // the level loop as one CUDA graph, and what it was built for
  cudaGraphExec_t gexec;
  uint64_t g_full;
  g3_msbfs_opts g_opts;
  g3_msbfs_stats last;  // of the last call
  unsigned long long* h_ctr;
  int32_t* d_roots;
  cudaEvent_t ev[2];
};

void g3_ms_ws_free(g3_ms_ws* w) {
  if (!w) return;
  void* all[] = {w->vis,   w->fa,   w->fb,    w->nx,  w->lv,     w->qa,
                 w->qb,    w->heavy, w->pend, w->items, w->ctr, w->d_roots};
  for (void* p : all)
    if (p) cudaFree(p);
  if (w->h_ctr) cudaFreeHost(w->h_ctr);
  for (int i = 0; i < 2; ++i)
    if (w->ev[i]) cudaEventDestroy(w->ev[i]);
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  free(w);
}

static g3_status ms_ws_create(g3_graph* g, g3_ms_ws** out) {
  g3_ms_ws* w = (g3_ms_ws*)calloc(1, sizeof(g3_ms_ws));
  if (!w) return G3_ENOMEM;
  w->nb = g->n_bfs;
  const size_t nb1 = (size_t)g->n_bfs + 4;
  // a row of d entries yields at most d / MS_CHUNK items
  w->items_cap = g->nnz / MS_CHUNK + 4;
  struct {
    void** p;
    size_t bytes;
  } req[] = {{(void**)&w->vis, nb1 * 8}, {(void**)&w->fa, nb1 * 8},   {(void**)&w->fb, nb1 * 8},
             {(void**)&w->nx, nb1 * 8},  {(void**)&w->lv, nb1 * 64},  {(void**)&w->qa, nb1 * 4},
             {(void**)&w->qb, nb1 * 4},  {(void**)&w->heavy, nb1 * 4}, {(void**)&w->ctr, MS_NCTR * 8},
             {(void**)&w->pend, nb1 * 4}, {(void**)&w->items, (size_t)w->items_cap * 8},
             {(void**)&w->d_roots, 64 * 4}};
  for (auto& r : req) {
    cudaError_t e = g3_alloc_should_fail() ? cudaErrorMemoryAllocation
                                            : cudaMalloc(r.p, r.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g3_set_error("g3_msbfs workspace: cudaMalloc(%zu): %s", r.bytes, cudaGetErrorString(e));
      g3_ms_ws_free(w);
      return G3_ENOMEM;
    }
  }
  if (cudaMallocHost((void**)&w->h_ctr, MS_NCTR * 8) != cudaSuccess ||
      cudaEventCreate(&w->ev[0]) != cudaSuccess || cudaEventCreate(&w->ev[1]) != cudaSuccess) {
    cudaGetLastError();
    g3_ms_ws_free(w);
    return G3_ENOMEM;
  }
  *out = w;
  return G3_OK;
}

// ---------------------------------------------------------------- kernels
// Seeds F and vis with the roots (BFS-graph labels) and queues each seed
// vertex once.
__global__ void ms_seed(const int32_t* roots, int k, const int32_t* new_of_old, int32_t nb,
                        uint64_t* vis, uint64_t* F, int8_t* lv, int32_t* q,
                        unsigned long long* ctr, const int64_t* off) {
  const int s = threadIdx.x;
  if (s >= k) return;
  const int32_t x = new_of_old ? new_of_old[roots[s]] : roots[s];
  if (x < 0 || x >= nb) return;
  const uint64_t old = atomicOr((unsigned long long*)&F[x], 1ull << s);
  atomicOr((unsigned long long*)&vis[x], 1ull << s);
  lv[(int64_t)x * 64 + s] = 0;
  if (old == 0) {
    const unsigned long long slot = atomicAdd(&ctr[0], 1ull);
    q[slot] = x;
    atomicAdd(&ctr[1], (unsigned long long)(off[x + 1] - off[x]));
  }
}

// Queues chunks 1 .. of a row longer than MS_CHUNK (warp-wide call).
__device__ __forceinline__ void ms_queue_chunks(int32_t v, int64_t deg, int2* items,
                                                unsigned long long* nitems, int lane) {
  const int64_t nch = (deg + MS_CHUNK - 1) / MS_CHUNK;
  if (nch <= 1) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(nitems, (unsigned long long)(nch - 1));
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int64_t c = 1 + lane; c < nch; c += 32) items[base + c - 1] = make_int2(v, (int32_t)c);
}

// Push of row entries [b, e) of frontier vertex u (warp-wide call):
// N[w] |= F[u] & ~vis[w]; first touchers of w queue it in `touched`.
__device__ __forceinline__ void ms_push_range(int64_t b, int64_t e, uint64_t fu,
                                              const int32_t* __restrict__ col,
                                              const uint64_t* __restrict__ vis, uint64_t* N,
                                              int32_t* touched, unsigned long long* tlen,
                                              int lane) {
  for (int64_t j0 = b; j0 < e; j0 += 32) {
    const int64_t j = j0 + lane;
    bool first = false;
    int32_t w = 0;
    if (j < e) {
      w = col[j];
      const uint64_t m = fu & ~__ldcg((const unsigned long long*)&vis[w]);
      if (m) {
        const uint64_t o = atomicOr((unsigned long long*)&N[w], m);
        first = (o == 0);
      }
    }
    g3_warp_append(0xffffffffu, first, w, touched, tlen);
  }
}

// Push, one warp per frontier vertex (first chunk of long rows).
__global__ void __launch_bounds__(256) ms_push(const int32_t* __restrict__ q,
                                               const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ col,
                                               const uint64_t* __restrict__ F,
                                               const uint64_t* __restrict__ vis, uint64_t* N,
                                               int32_t* touched, unsigned long long* ctr,
                                               int2* items) {
  const int64_t qlen = (int64_t)ctr[MS_QCUR];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < qlen; i += nwarps) {
    const int32_t u = q[i];
    const uint64_t fu = F[u];
    const int64_t b = off[u], e = off[u + 1];
    ms_queue_chunks(u, e - b, items, &ctr[3], lane);
    ms_push_range(b, min(e, b + MS_CHUNK), fu, col, vis, N, touched, &ctr[2], lane);
  }
}

// Push of the queued chunks, one warp per (vertex, chunk) item.
__global__ void __launch_bounds__(256) ms_push_chunks(const int2* __restrict__ items,
                                                      const int64_t* __restrict__ off,
                                                      const int32_t* __restrict__ col,
                                                      const uint64_t* __restrict__ F,
                                                      const uint64_t* __restrict__ vis,
                                                      uint64_t* N, int32_t* touched,
                                                      unsigned long long* ctr) {
  const int64_t len = (int64_t)ctr[3];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < len; i += nwarps) {
    const int2 it = items[i];
    const int64_t b = off[it.x] + (int64_t)it.y * MS_CHUNK;
    ms_push_range(b, min(off[it.x + 1], b + MS_CHUNK), F[it.x], col, vis, N, touched, &ctr[2],
                  lane);
  }
}

// The four level bytes of a 32-bit word whose sources are set in nib (bit i
// -> byte i) become lnext (rep: lnext in every byte); the others stay.
__device__ __forceinline__ uint32_t ms_merge4(uint32_t old, uint32_t nib, uint32_t rep) {
  const uint32_t m = __vcmpne4((nib * 0x01010101u) & 0x08040201u, 0u);
  return (old & ~m) | (rep & m);
}

// Records v's new source bits at level lnext: a few bits as single bytes;
// more as 16-byte read-merge-writes of the 16-source quarters of v's 64-byte
// row that have new bits (one store per quarter instead of one per source).
// One thread owns v's row at a time (v is taken by one kernel of a level).
__device__ __forceinline__ void ms_take(int32_t v, uint64_t nv, uint64_t* vis, uint64_t vv,
                                        int8_t* lv, int8_t lnext) {
  vis[v] = vv | nv;
  if (__popcll((long long)nv) <= 4) {
    uint64_t bits = nv;
    while (bits) {
      const int s = __ffsll((long long)bits) - 1;
      lv[(int64_t)v * 64 + s] = lnext;
      bits &= bits - 1;
    }
    return;
  }
  int4* row = reinterpret_cast<int4*>(lv + (int64_t)v * 64);
  const uint32_t rep = 0x01010101u * (uint32_t)(uint8_t)lnext;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t b16 = (uint32_t)(nv >> (16 * q)) & 0xFFFFu;
    if (!b16) continue;
    int4 w = row[q];
    w.x = (int)ms_merge4((uint32_t)w.x, b16 & 0xFu, rep);
    w.y = (int)ms_merge4((uint32_t)w.y, (b16 >> 4) & 0xFu, rep);
    w.z = (int)ms_merge4((uint32_t)w.z, (b16 >> 8) & 0xFu, rep);
    w.w = (int)ms_merge4((uint32_t)w.w, (b16 >> 12) & 0xFu, rep);
    row[q] = w;
  }
}

// Finalize after a push: keep N[w]'s bits not yet in vis[w] as the new
// frontier word, record their levels, queue w when anything is new, clear N.
__global__ void ms_push_finalize(const int32_t* __restrict__ touched, uint64_t* N,
                                 uint64_t* vis, uint64_t* Fn, int8_t* lv, int32_t* qn,
                                 const int64_t* __restrict__ off, unsigned long long* ctr) {
  const int64_t len = (int64_t)ctr[2];
  const int8_t lnext = (int8_t)ctr[MS_LNEXT];
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < len;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool want = false;
    int32_t w = 0;
    unsigned long long d = 0;
    if (i < len) {
      w = touched[i];
      const uint64_t nw = N[w];
      N[w] = 0;
      const uint64_t vw = vis[w];
      const uint64_t nv = nw & ~vw;
      Fn[w] = nv;
      if (nv) {
        ms_take(w, nv, vis, vw, lv, lnext);
        want = true;
        d = (unsigned long long)(off[w + 1] - off[w]);
      }
    }
    g3_warp_append(0xffffffffu, want, w, qn, &ctr[0]);
    for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0 && d) atomicAdd(&ctr[1], d);
  }
}

// Pull: thread per vertex for degree < heavy_deg, else queued for ms_pull_heavy.
__global__ void __launch_bounds__(256) ms_pull(int32_t nb, const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ col,
                                               const uint64_t* __restrict__ F, uint64_t* vis,
                                               uint64_t* Fn, int8_t* lv, uint64_t full,
                                               int64_t heavy_deg, int32_t* heavy, int32_t* qn,
                                               unsigned long long* ctr) {
  const int8_t lnext = (int8_t)ctr[MS_LNEXT];
  const bool col_al16 = ((uintptr_t)col & 15) == 0;
  unsigned long long rd_all = 0, sc_all = 0;  // work counts, added once per warp
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nb;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    bool want = false, big = false;
    unsigned long long d = 0;
    if (v < nb) {
      const uint64_t vv = vis[v];
      uint64_t nv = 0;
      if (vv != full) {
        const int64_t b = off[v], e = off[v + 1];
        if (e - b >= heavy_deg) {
          big = true;
        } else {
          sc_all += 1;
          // up to the next multiple of 4 one entry at a time, then two
          // 128-bit column loads and eight independent gathers per step
          // (four near the row's end); the
          // exit test runs per step (vector loads only on a 16-byte aligned
          // col, which the allocator gives)
          uint64_t acc = 0;
          int64_t j = b;
          for (; j < e && (j & 3) && (acc | vv) != full; ++j) acc |= __ldg(&F[col[j]]);
          for (; col_al16 && j + 8 <= e && (acc | vv) != full; j += 8) {
            const int4 c4 = __ldg(reinterpret_cast<const int4*>(col + j));
            const int4 c5 = __ldg(reinterpret_cast<const int4*>(col + j + 4));
            acc |= ((__ldg(&F[c4.x]) | __ldg(&F[c4.y])) | (__ldg(&F[c4.z]) | __ldg(&F[c4.w]))) |
                   ((__ldg(&F[c5.x]) | __ldg(&F[c5.y])) | (__ldg(&F[c5.z]) | __ldg(&F[c5.w])));
          }
          for (; col_al16 && j + 4 <= e && (acc | vv) != full; j += 4) {
            const int4 c4 = __ldg(reinterpret_cast<const int4*>(col + j));
            acc |= (__ldg(&F[c4.x]) | __ldg(&F[c4.y])) | (__ldg(&F[c4.z]) | __ldg(&F[c4.w]));
          }
          for (; j < e && (acc | vv) != full; ++j) acc |= __ldg(&F[col[j]]);
          rd_all += (unsigned long long)(j - b);
          nv = acc & ~vv;
          if (nv) {
            ms_take((int32_t)v, nv, vis, vv, lv, lnext);
            want = true;
            d = (unsigned long long)(e - b);
          }
        }
      }
      if (!big) Fn[v] = nv;
    }
    g3_warp_append(0xffffffffu, big, (int32_t)v, heavy, &ctr[2]);
    g3_warp_append(0xffffffffu, want, (int32_t)v, qn, &ctr[0]);
    for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0 && d) atomicAdd(&ctr[1], d);
  }
  for (int o = 16; o; o >>= 1) {
    rd_all += __shfl_xor_sync(0xffffffffu, rd_all, o);
    sc_all += __shfl_xor_sync(0xffffffffu, sc_all, o);
  }
  if ((threadIdx.x & 31) == 0 && sc_all) {
    atomicAdd(&ctr[5], rd_all);
    atomicAdd(&ctr[6], sc_all);
  }
}

// Frontier sources among row entries [b, e) (warp-wide call): the OR of
// F over the entries, cut short once `have` | the OR covers every source.
__device__ __forceinline__ uint64_t ms_pull_range(int64_t b, int64_t e, uint64_t have,
                                                  uint64_t full,
                                                  const int32_t* __restrict__ col,
                                                  const uint64_t* __restrict__ F, int lane,
                                                  int64_t& read) {
  uint64_t acc = 0;
  for (int64_t j0 = b; j0 < e; j0 += 32) {
    const int64_t j = j0 + lane;
    uint64_t x = j < e ? __ldg(&F[col[j]]) : 0ull;
    read += e - j0 < 32 ? e - j0 : 32;
    for (int o = 16; o; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
    acc |= x;
    if ((acc | have) == full) break;
  }
  return acc;
}

// Queues a vertex that found new sources for the next level.
__device__ __forceinline__ void ms_emit(int32_t v, uint64_t nv, uint64_t vv, uint64_t* vis,
                                        uint64_t* Fn, int8_t* lv, int8_t lnext, int32_t* qn,
                                        int64_t deg, unsigned long long* ctr) {
  Fn[v] = nv;
  if (nv) {
    ms_take(v, nv, vis, vv, lv, lnext);
    const unsigned long long slot = atomicAdd(&ctr[0], 1ull);
    qn[slot] = v;
    atomicAdd(&ctr[1], (unsigned long long)deg);
  }
}

// Pull for high-degree vertices: one warp per vertex over the row's first
// chunk; a row longer than that, still missing sources, has its other
// chunks queued and its partial OR parked in N[v] for ms_pull_pending.
__global__ void __launch_bounds__(256) ms_pull_heavy(const int32_t* __restrict__ heavy,
                                                     const int64_t* __restrict__ off,
                                                     const int32_t* __restrict__ col,
                                                     const uint64_t* __restrict__ F,
                                                     uint64_t* vis, uint64_t* Fn, uint64_t* N,
                                                     int8_t* lv, uint64_t full, int32_t* qn,
                                                     int32_t* pend, int2* items,
                                                     unsigned long long* ctr) {
  const int64_t len = (int64_t)ctr[2];
  const int8_t lnext = (int8_t)ctr[MS_LNEXT];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t read = 0, scanned = 0;  // work counts, added once per warp
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < len; i += nwarps) {
    const int32_t v = heavy[i];
    const uint64_t vv = vis[v];
    const int64_t b = off[v], e = off[v + 1];
    const uint64_t acc = ms_pull_range(b, min(e, b + MS_CHUNK), vv, full, col, F, lane, read);
    ++scanned;
    if (e - b > MS_CHUNK && (acc | vv) != full) {
      ms_queue_chunks(v, e - b, items, &ctr[3], lane);
      if (lane == 0) {
        N[v] = acc;
        pend[atomicAdd(&ctr[4], 1ull)] = v;
      }
    } else if (lane == 0) {
      ms_emit(v, acc & ~vv, vv, vis, Fn, lv, lnext, qn, e - b, ctr);
    }
  }
  if (lane == 0 && scanned) {
    atomicAdd(&ctr[5], (unsigned long long)read);
    atomicAdd(&ctr[6], (unsigned long long)scanned);
  }
}

// Pull of the queued chunks, one warp per item; partial ORs meet in N[v].
__global__ void __launch_bounds__(256) ms_pull_chunks(const int2* __restrict__ items,
                                                      const int64_t* __restrict__ off,
                                                      const int32_t* __restrict__ col,
                                                      const uint64_t* __restrict__ F,
                                                      const uint64_t* __restrict__ vis,
                                                      uint64_t* N, uint64_t full,
                                                      unsigned long long* ctr) {
  const int64_t len = (int64_t)ctr[3];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t read = 0;  // entries read, added once per warp
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < len; i += nwarps) {
    const int2 it = items[i];
    const int64_t b = off[it.x] + (int64_t)it.y * MS_CHUNK;
    const uint64_t acc = ms_pull_range(b, min(off[it.x + 1], b + MS_CHUNK), vis[it.x], full,
                                       col, F, lane, read);
    if (lane == 0 && acc) atomicOr((unsigned long long*)&N[it.x], acc);
  }
  if (lane == 0 && read) atomicAdd(&ctr[5], (unsigned long long)read);
}

// Finishes the split heavy vertices: new sources = N[v] & ~vis[v]; N cleared.
__global__ void ms_pull_pending(const int32_t* __restrict__ pend, const int64_t* __restrict__ off,
                                uint64_t* vis, uint64_t* Fn, uint64_t* N, int8_t* lv, int32_t* qn,
                                unsigned long long* ctr) {
  const int64_t len = (int64_t)ctr[4];
  const int8_t lnext = (int8_t)ctr[MS_LNEXT];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = pend[i];
    const uint64_t vv = vis[v];
    const uint64_t acc = N[v];
    N[v] = 0;
    ms_emit(v, acc & ~vv, vv, vis, Fn, lv, lnext, qn, off[v + 1] - off[v], ctr);
  }
}

// level[s][o] for s < k over tiles of MS_OUT_TILE original IDs: gather the
// 64-byte rows of the tile's vertices into shared memory (a level is valid
// where the source's bit is set in vis), then write each source's slice of
// the tile as 32-bit words, one 128-byte run per warp store.
#define MS_OUT_TILE 128
__global__ void __launch_bounds__(256) ms_out(int32_t n, int32_t nb, int k,
                                              const int32_t* __restrict__ new_of_old,
                                              const uint64_t* __restrict__ vis,
                                              const int8_t* __restrict__ lv, int8_t* level) {
  __shared__ __align__(16) int8_t tile[MS_OUT_TILE][64 + 4];
  __shared__ int32_t xs[MS_OUT_TILE];
  __shared__ uint64_t vm[MS_OUT_TILE];
  const int64_t ntiles = ((int64_t)n + MS_OUT_TILE - 1) / MS_OUT_TILE;
  const bool aligned = ((uintptr_t)level & 3) == 0 && (n & 3) == 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t o0 = t * MS_OUT_TILE;
    if (threadIdx.x < MS_OUT_TILE) {
      const int64_t o = o0 + threadIdx.x;
      int32_t x = -1;
      if (o < n) x = new_of_old ? new_of_old[o] : (int32_t)o;
      if (x >= nb) x = -1;
      xs[threadIdx.x] = x;
      vm[threadIdx.x] = x >= 0 ? vis[x] : 0ull;
    }
    __syncthreads();
    // MS_OUT_TILE rows x 4 quarters of 16 bytes, two per thread
#pragma unroll
    for (int h = 0; h < (MS_OUT_TILE * 4) / 256; ++h) {
      const int idx = threadIdx.x + h * 256;
      const int r = idx >> 2, qd = idx & 3;
      const int32_t x = xs[r];
      int4 val = make_int4(-1, -1, -1, -1);
      if (x >= 0) val = *reinterpret_cast<const int4*>(lv + (int64_t)x * 64 + qd * 16);
      // bytes of sources not reached become -1, four at a time
      const uint32_t nb16 = ~(uint32_t)(vm[r] >> (qd * 16)) & 0xFFFFu;
      uint32_t* trow = reinterpret_cast<uint32_t*>(&tile[r][qd * 16]);
      trow[0] = ms_merge4((uint32_t)val.x, nb16 & 0xFu, 0xFFFFFFFFu);
      trow[1] = ms_merge4((uint32_t)val.y, (nb16 >> 4) & 0xFu, 0xFFFFFFFFu);
      trow[2] = ms_merge4((uint32_t)val.z, (nb16 >> 8) & 0xFu, 0xFFFFFFFFu);
      trow[3] = ms_merge4((uint32_t)val.w, (nb16 >> 12) & 0xFu, 0xFFFFFFFFu);
    }
    __syncthreads();
    constexpr int WPT = MS_OUT_TILE / 4;  // 32-bit words per source per tile
    for (int idx = threadIdx.x; idx < k * WPT; idx += blockDim.x) {
      const int sidx = idx / WPT, c = idx % WPT;
      const int64_t o = o0 + 4 * c;
      int8_t* dst = level + (int64_t)sidx * n + o;
      if (aligned && o + 3 < n) {
        const uint32_t w = (uint32_t)(uint8_t)tile[4 * c][sidx] |
                           ((uint32_t)(uint8_t)tile[4 * c + 1][sidx] << 8) |
                           ((uint32_t)(uint8_t)tile[4 * c + 2][sidx] << 16) |
                           ((uint32_t)(uint8_t)tile[4 * c + 3][sidx] << 24);
        *reinterpret_cast<uint32_t*>(dst) = w;
      } else {
        for (int j = 0; j < 4 && o + j < n; ++j) dst[j] = tile[4 * c + j][sidx];
      }
    }
    __syncthreads();
  }
}

// The roots themselves (also isolated roots, which are not in the BFS graph).
__global__ void ms_roots_out(const int32_t* roots, int k, int32_t n, int8_t* level) {
  const int s = threadIdx.x;
  if (s < k) level[(int64_t)s * n + roots[s]] = 0;
}

// ------------------------------------------------------ level loop graph
// Before each level: reads the frontier produced by the previous one, ends
// the loop when it is empty (or flags a level above 126), else chooses pull
// (sum of frontier degrees * push_alpha > nnz) or push, keeps the per-call
// counts, clears the per-level counters and selects the SWITCH branch.
__global__ void ms_control(unsigned long long* ctr, int64_t nnz, int32_t push_alpha,
                           cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_kind) {
  const unsigned long long qlen = ctr[0], mf = ctr[1], L = ctr[MS_LEVEL];
  if (qlen == 0 || L >= 127) {
    if (qlen != 0) ctr[MS_ERANGE] = 1;  // expanding level 127 would write level 128
    cudaGraphSetConditional(h_kind, 2u);  // no branch
    cudaGraphSetConditional(h_loop, 0u);
    return;
  }
  const bool pull = (long long)mf * (long long)push_alpha > nnz;
  if (pull) {
    ctr[MS_PULLS] += 1;
  } else {
    ctr[MS_PUSHES] += 1;
    ctr[MS_PUSHED] += mf;  // every row entry of the frontier is pushed
  }
  ctr[MS_QCUR] = qlen;
  ctr[MS_LNEXT] = L + 1;
  ctr[MS_LEVEL] = L + 1;
  for (int i = 0; i < 5; ++i) ctr[i] = 0;
  cudaGraphSetConditional(h_kind, pull ? 0u : 1u);
  cudaGraphSetConditional(h_loop, 1u);
}

// Push needs Fn zero outside the new frontier.
__global__ void ms_clear(uint64_t* Fn, int32_t nb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nb;
       i += (int64_t)gridDim.x * blockDim.x)
    Fn[i] = 0;
}

static g3_status ms_add_kernel(cudaGraph_t gr, cudaGraphNode_t* node, cudaGraphNode_t* dep,
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

struct MsNodeParams {
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  MsNodeParams() { memset(raw, 0, sizeof(raw)); }
  cudaGraphNodeParams& get() { return *reinterpret_cast<cudaGraphNodeParams*>(raw); }
};

// The level loop of one call as a CUDA graph: WHILE { control -> SWITCH
// {pull, push} for a level from (fa, qa) into (fb, qb), then the same for a
// level from (fb, qb) into (fa, qa) }. Kernel arguments are fixed; what
// changes per level lives in ctr.
static g3_status ms_build_graph(g3_graph* g, g3_ms_ws* w, uint64_t full, const g3_msbfs_opts& o) {
  cudaGraph_t top = nullptr;
  G3_TRY_CUDA(cudaGraphCreate(&top, 0));
  g3_status st = G3_OK;
  const int grid = G3_NUM_SMS * 8;
  int32_t nb = w->nb;
  int64_t nnz = g->nnz, heavy_deg = o.pull_warp_deg;
  int32_t push_alpha = o.push_alpha;
  const int64_t* off = g->off;
  const int32_t* col = g->col;
  uint64_t f = full;
  cudaGraphConditionalHandle h_loop, h_kind[2];
  // per half: the frontier buffers it reads and writes
  uint64_t* Fs[2][2] = {{w->fa, w->fb}, {w->fb, w->fa}};
  int32_t* Qs[2][2] = {{w->qa, w->qb}, {w->qb, w->qa}};
  do {
    if (cudaGraphConditionalHandleCreate(&h_loop, top, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess) { st = G3_ECUDA; break; }
    MsNodeParams wb;
    cudaGraphNodeParams& wp = wb.get();
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp) != cudaSuccess) {
      st = G3_ECUDA;
      break;
    }
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    for (int half = 0; half < 2 && st == G3_OK; ++half) {
      if (cudaGraphConditionalHandleCreate(&h_kind[half], body, 0, 0) != cudaSuccess) {
        st = G3_ECUDA;
        break;
      }
    }
    if (st != G3_OK) break;
    // argument storage must outlive cudaGraphAddKernelNode only (copied in)
    for (int half = 0; half < 2 && st == G3_OK; ++half) {
      uint64_t *F = Fs[half][0], *Fn = Fs[half][1];
      int32_t *q = Qs[half][0], *qn = Qs[half][1];
      cudaGraphNode_t ctl, sw;
      void* a_ctl[] = {&w->ctr, &nnz, &push_alpha, &h_loop, &h_kind[half]};
      if ((st = ms_add_kernel(body, &ctl, half ? &prev : nullptr, (void*)ms_control, 1, 1,
                              a_ctl)))
        break;
      MsNodeParams sb;
      cudaGraphNodeParams& sp = sb.get();
      sp.type = cudaGraphNodeTypeConditional;
      sp.conditional.handle = h_kind[half];
      sp.conditional.type = cudaGraphCondTypeSwitch;
      sp.conditional.size = 2;
      if (cudaGraphAddNode(&sw, body, &ctl, nullptr, 1, &sp) != cudaSuccess) {
        st = G3_ECUDA;
        break;
      }
      cudaGraph_t pull = sp.conditional.phGraph_out[0], push = sp.conditional.phGraph_out[1];
      cudaGraphNode_t n0, n1, n2, n3;
      void* a_pull[] = {&nb, &off, &col, &F, &w->vis, &Fn, &w->lv, &f, &heavy_deg, &w->heavy,
                        &qn, &w->ctr};
      void* a_heavy[] = {&w->heavy, &off, &col, &F, &w->vis, &Fn, &w->nx, &w->lv, &f, &qn,
                         &w->pend, &w->items, &w->ctr};
      void* a_chunks[] = {&w->items, &off, &col, &F, &w->vis, &w->nx, &f, &w->ctr};
      void* a_pend[] = {&w->pend, &off, &w->vis, &Fn, &w->nx, &w->lv, &qn, &w->ctr};
      if ((st = ms_add_kernel(pull, &n0, nullptr, (void*)ms_pull, grid, 256, a_pull))) break;
      if ((st = ms_add_kernel(pull, &n1, &n0, (void*)ms_pull_heavy, grid, 256, a_heavy))) break;
      if ((st = ms_add_kernel(pull, &n2, &n1, (void*)ms_pull_chunks, grid, 256, a_chunks)))
        break;
      if ((st = ms_add_kernel(pull, &n3, &n2, (void*)ms_pull_pending, G3_NUM_SMS, 256, a_pend)))
        break;
      void* a_clear[] = {&Fn, &nb};
      void* a_push[] = {&q, &off, &col, &F, &w->vis, &w->nx, &w->heavy, &w->ctr, &w->items};
      void* a_pchunks[] = {&w->items, &off, &col, &F, &w->vis, &w->nx, &w->heavy, &w->ctr};
      void* a_fin[] = {&w->heavy, &w->nx, &w->vis, &Fn, &w->lv, &qn, &off, &w->ctr};
      if ((st = ms_add_kernel(push, &n0, nullptr, (void*)ms_clear, grid, 256, a_clear))) break;
      if ((st = ms_add_kernel(push, &n1, &n0, (void*)ms_push, grid, 256, a_push))) break;
      if ((st = ms_add_kernel(push, &n2, &n1, (void*)ms_push_chunks, grid, 256, a_pchunks)))
        break;
      if ((st = ms_add_kernel(push, &n3, &n2, (void*)ms_push_finalize, grid, 256, a_fin))) break;
      prev = sw;
    }
    if (st != G3_OK) break;
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, top, 0) != cudaSuccess) {
      st = G3_ECUDA;
      break;
    }
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    w->gexec = ex;
    w->g_full = full;
    w->g_opts = o;
  } while (0);
  if (st != G3_OK) {
    cudaError_t e = cudaGetLastError();
    g3_set_error("g3_msbfs: building the level-loop graph failed: %s", cudaGetErrorString(e));
  }
  cudaGraphDestroy(top);
  return st;
}

// ------------------------------------------------------------------ host
extern "C" void g3_msbfs_opts_default(g3_msbfs_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->push_alpha = 14;
  o->pull_warp_deg = 256;
}

extern "C" g3_status g3_msbfs(g3_graph* g, const int32_t* roots, int32_t k,
                              const g3_msbfs_opts* opts, int8_t* level, int32_t* n_levels,
                              float* ms, void* stream) {
  if (!g || !roots || !level || k < 1 || k > 64) {
    g3_set_error("g3_msbfs: bad arguments (k must be 1..64)");
    return G3_EINVAL;
  }
  for (int s = 0; s < k; ++s)
    if (roots[s] < 0 || roots[s] >= g->n) {
      g3_set_error("g3_msbfs: root %d outside [0, %d)", roots[s], g->n);
      return G3_EINVAL;
    }
  g3_msbfs_opts o;
  if (opts) o = *opts; else g3_msbfs_opts_default(&o);
  if (o.push_alpha <= 0 || o.pull_warp_deg < 1) {
    g3_set_error("g3_msbfs: bad options");
    return G3_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!g->ms) G3_TRY(ms_ws_create(g, &g->ms));
  g3_ms_ws* w = g->ms;
  const int32_t nb = w->nb;
  const uint64_t full = k == 64 ? ~0ull : ((1ull << k) - 1ull);
  const int32_t* n2o = g->relabelled ? g->new_of_old : nullptr;
  unsigned long long* h = w->h_ctr;
  const int grid = G3_NUM_SMS * 8;

  if (w->items_cap < g->nnz / MS_CHUNK + 4) {
    g3_set_error("g3_msbfs: workspace does not fit the graph");
    return G3_ESTATE;
  }
  if (!w->gexec || w->g_full != full || w->g_opts.push_alpha != o.push_alpha ||
      w->g_opts.pull_warp_deg != o.pull_warp_deg)
    G3_TRY(ms_build_graph(g, w, full, o));
  G3_TRY_CUDA(cudaEventRecord(w->ev[0], s));
  G3_TRY_CUDA(cudaMemcpyAsync(w->d_roots, roots, (size_t)k * 4, cudaMemcpyHostToDevice, s));
  G3_TRY_CUDA(cudaMemsetAsync(w->vis, 0, (size_t)nb * 8 + 8, s));
  G3_TRY_CUDA(cudaMemsetAsync(w->fa, 0, (size_t)nb * 8 + 8, s));
  G3_TRY_CUDA(cudaMemsetAsync(w->nx, 0, (size_t)nb * 8 + 8, s));
  G3_TRY_CUDA(cudaMemsetAsync(w->ctr, 0, MS_NCTR * 8, s));
  ms_seed<<<1, 64, 0, s>>>(w->d_roots, k, n2o, nb, w->vis, w->fa, w->lv, w->qa, w->ctr, g->off);
  G3_CHECK_LAUNCH();
  // the whole level loop: one graph launch, no host round trip per level
  G3_TRY_CUDA(cudaGraphLaunch(w->gexec, s));
  ms_out<<<grid, 256, 0, s>>>(g->n, nb, k, n2o, w->vis, w->lv, level);
  G3_CHECK_LAUNCH();
  ms_roots_out<<<1, 64, 0, s>>>(w->d_roots, k, g->n, level);
  G3_CHECK_LAUNCH();
  G3_TRY_CUDA(cudaEventRecord(w->ev[1], s));
  G3_TRY_CUDA(cudaMemcpyAsync(h, w->ctr, MS_NCTR * 8, cudaMemcpyDeviceToHost, s));
  G3_TRY_CUDA(cudaStreamSynchronize(s));
  if (h[MS_ERANGE]) {
    g3_set_error("g3_msbfs: a level exceeds 126, the int8 range of the output");
    return G3_ERANGE;
  }
  const int32_t L = (int32_t)h[MS_LEVEL];
  if (n_levels) *n_levels = L;
  if (ms) cudaEventElapsedTime(ms, w->ev[0], w->ev[1]);
  g3_msbfs_stats stats;
  memset(&stats, 0, sizeof(stats));
  stats.levels = L;
  stats.pull_levels = (int32_t)h[MS_PULLS];
  stats.push_levels = (int32_t)h[MS_PUSHES];
  stats.push_entries = (int64_t)h[MS_PUSHED];
  stats.pull_entries = (int64_t)h[5];
  stats.pull_vertices = (int64_t)h[6];
  w->last = stats;
  return G3_OK;
}

extern "C" g3_status g3_msbfs_last_stats(const g3_graph* g, g3_msbfs_stats* out) {
  if (!g || !out) {
    g3_set_error("g3_msbfs_last_stats: null argument");
    return G3_EINVAL;
  }
  if (!g->ms) {
    g3_set_error("g3_msbfs_last_stats: no multi-source search has run on this graph");
    return G3_ESTATE;
  }
  *out = g->ms->last;
  return G3_OK;
}
