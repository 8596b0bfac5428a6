// Graph accessors and lifetime.
#include <stdlib.h>

#include "g3_internal.cuh"

extern "C" g3_status g3_graph_info_get(const g3_graph* g, g3_graph_info* info) {
  if (!g || !info) {
    g3_set_error("g3_graph_info_get: null argument");
    return G3_EINVAL;
  }
  info->n = g->n;
  info->n_bfs = g->n_bfs;
  info->n_plus = g->relabelled ? g->n_plus : -1;
  info->relabelled = g->relabelled;
  info->nnz = g->nnz;
  info->max_degree = g->max_degree;
  return G3_OK;
}

extern "C" g3_status g3_get_perm(const g3_graph* g, int32_t* old_of_new, int32_t* new_of_old,
                                 void* stream) {
  if (!g) {
    g3_set_error("g3_get_perm: graph is NULL");
    return G3_EINVAL;
  }
  if (!g->relabelled) {
    g3_set_error("g3_get_perm: graph is not relabelled");
    return G3_ESTATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)g->n * sizeof(int32_t);
  if (old_of_new)
    G3_TRY_CUDA(cudaMemcpyAsync(old_of_new, g->old_of_new, bytes, cudaMemcpyDefault, s));
  if (new_of_old)
    G3_TRY_CUDA(cudaMemcpyAsync(new_of_old, g->new_of_old, bytes, cudaMemcpyDefault, s));
  return G3_OK;
}

extern "C" g3_status g3_get_csr(const g3_graph* g, int64_t* off, int32_t* col, void* stream) {
  if (!g) {
    g3_set_error("g3_get_csr: graph is NULL");
    return G3_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (off)
    G3_TRY_CUDA(cudaMemcpyAsync(off, g->off, ((size_t)g->n_bfs + 1) * sizeof(int64_t),
                                cudaMemcpyDefault, s));
  if (col && g->nnz > 0)
    G3_TRY_CUDA(cudaMemcpyAsync(col, g->col, (size_t)g->nnz * sizeof(int32_t),
                                cudaMemcpyDefault, s));
  return G3_OK;
}

extern "C" void g3_graph_free(g3_graph* g) {
  if (!g) return;
  // the graph's arrays were allocated stream-ordered on the callers'
  // streams; waiting for the device first orders the frees after any work
  // still reading them, whatever stream it was queued on
  cudaDeviceSynchronize();
  cudaGetLastError();
  if (g->ws) g3_bfs_ws_free(g->ws);
  if (g->ms) g3_ms_ws_free(g->ms);
  void* all[] = {g->off, g->col, g->old_of_new, g->new_of_old, g->comp_rng};
  for (void* p : all)
    if (p) cudaFreeAsync(p, 0);
  cudaStreamSynchronize(0);
  free(g);
}
