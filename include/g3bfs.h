/*
 * g3bfs -- C ABI of the GB300 (sm_103a) library for breadth-first search on
 * RCM-relabelled graphs (Jiang et al., "Fast and Efficient Parallel
 * Breadth-First Search with Power-law Graph Transformation", PPoPP'21).
 *
 * Problem statement (Sec. 2.1): given an undirected, unweighted graph
 * G = (V, E) and a source s, produce the predecessor map pi with pi(s) = s,
 * pi(v) = -1 when v is unreachable, and every level-k vertex discovered before
 * any level-(k+1) vertex. The library also returns level[] (hop distance).
 *
 * Pipeline: g3_build_csr (Sec. 3.1) -> g3_rcm_relabel (Algorithm 3, Sec. 3.2)
 * -> g3_bfs (Algorithm 2 with per-level direction choice; top-down as
 * Algorithms 1/4, bottom-up as Algorithm 5) -> parent[] / level[] in original
 * vertex IDs.
 *
 * Conventions for every call:
 *   - Vertex IDs are int32 in [0, n). Edge counts and CSR offsets are int64.
 *   - "device pointer" = memory the current CUDA device can address (e.g. a
 *     torch CUDA tensor's data_ptr()); "host pointer" = ordinary host memory.
 *     Where a call accepts either, it says so and finds out which it got.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is stream-ordered. Calls that must read a device-side
 *     count to size an allocation or to steer a loop synchronise the stream
 *     before returning; each call states whether it does.
 *   - Every call returns a g3_status. Calls never abort, trap or print;
 *     g3_status_str() gives a message, g3_last_error_detail() the detail of
 *     the last failure on the calling thread.
 *   - Outputs are caller-owned unless stated. The library owns a g3_graph and
 *     all device memory behind it until g3_graph_free().
 *   - A g3_graph is not thread-safe: run one call on it at a time.
 */
#ifndef G3BFS_H
#define G3BFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  G3_OK = 0,
  G3_EINVAL = 1,   /* bad argument: null pointer, size or ID out of range */
  G3_ENOMEM = 2,   /* a device or pinned-host allocation failed */
  G3_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  G3_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  G3_ERANGE = 5,   /* a result does not fit the requested output type */
  G3_ESTATE = 6    /* call not valid in the graph's current state */
} g3_status;

const char* g3_status_str(g3_status s);
/* Text of the last failure seen by a g3_* call on this thread ("" if none). */
const char* g3_last_error_detail(void);
/* Library version, e.g. "g3bfs 0.1 sm_103a". */
const char* g3_version(void);
/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices); for instrumentation. */
uint64_t g3_kernel_launches(void);

typedef struct g3_graph g3_graph;

typedef struct {
  int32_t n;          /* vertices of the input (original IDs 0..n-1) */
  int32_t n_bfs;      /* vertices the BFS graph has: n_plus if relabelled, else n */
  int32_t n_plus;     /* |V+|, non-isolated vertices (Sec. 3.2) */
  int32_t relabelled; /* 1 after g3_rcm_relabel */
  int64_t nnz;        /* directed CSR entries (each undirected edge twice) */
  int64_t max_degree;
} g3_graph_info;

/* Builds the cleaned CSR of the undirected graph given by m generated tuples
 * (src[i], dst[i]) (Sec. 3.1, Eq. 2; both directions stored, Sec. 3.1).
 * Self-loops and duplicate tuples are removed (the Graph500 generator emits
 * both, Sec. 4.2); degree(v) is then the row length. Rows are ascending.
 *   src, dst : device pointers, m int32 entries each, values in [0, n);
 *              read only; the caller keeps ownership.
 *   m        : number of tuples, >= 0.   n : vertices, 1 <= n < 2^31.
 *   out      : receives a new graph owned by the caller (g3_graph_free).
 * Synchronises `stream` (the entry count sizes an allocation).
 * Errors: G3_EINVAL (null pointer, n or m out of range, an endpoint outside
 * [0, n)), G3_ENOMEM, G3_ECUDA. On error *out is NULL. */
g3_status g3_build_csr(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                       void* stream, g3_graph** out);

/* Relabels the graph by Reverse Cuthill-McKee, Algorithm 3 (Sec. 3.2), in
 * place: V+ in increasing degree, neighbours visited in increasing degree,
 * each component started from its first unvisited vertex of V+ (the minimal
 * degree, Sec. 3.2), the Cuthill-McKee order reversed, isolated vertices
 * appended in ascending original ID and dropped from the BFS graph.
 * Ties in degree are broken by ascending original ID. The result equals the
 * serial algorithm exactly; on the GPU it is computed level-synchronously
 * (level k+1 of a component ordered by the position of its earliest-placed
 * neighbour in level k, then degree, then ID).
 * After the call the graph's CSR is the relabelled one over n_plus vertices
 * (rows ascending) and the permutation is kept for g3_bfs and g3_get_perm.
 * Each component's vertices get consecutive labels (a component is finished
 * before the next start is taken), and the label range of every vertex's
 * component is kept too (8 bytes per vertex of V+): g3_bfs's output pass
 * takes the reached set from its root's range instead of the visited bitmap.
 * Synchronises `stream`. Errors: G3_ESTATE (already relabelled), G3_ENOMEM,
 * G3_ECUDA. */
g3_status g3_rcm_relabel(g3_graph* g, void* stream);

/* Partial RCM (Sec. 4.6): reorders only the top p of V+ to cut the
 * relabelling cost. The paper gives no procedure; here the top
 * k = ceil(p_permille * n_plus / 1000) vertices are the last k of V+ in
 * (degree, ID) order, Algorithm 3 runs on that set alone (edges leaving it
 * ignored, the graph's degrees as ordering key) and its reverse order takes
 * labels 0..k-1; the rest of V+ takes labels k..n_plus-1 in ascending
 * original ID; isolated vertices follow as in g3_rcm_relabel, which is
 * p_permille = 1000. Afterwards the graph is relabelled exactly as after
 * g3_rcm_relabel (n_plus rows, permutation kept). Synchronises `stream`.
 * Errors: G3_EINVAL (p_permille outside [0, 1000]), G3_ESTATE, G3_ENOMEM,
 * G3_ECUDA. */
g3_status g3_rcm_relabel_partial(g3_graph* g, int32_t p_permille, void* stream);

g3_status g3_graph_info_get(const g3_graph* g, g3_graph_info* info);

/* Copies the permutation (device pointers, n entries each; either may be
 * NULL): old_of_new[new label] = original ID, new_of_old[original ID] = new
 * label. Labels [0, n_plus) are V+ in RCM order, [n_plus, n) the isolated
 * vertices. G3_ESTATE when the graph is not relabelled. Asynchronous. */
g3_status g3_get_perm(const g3_graph* g, int32_t* old_of_new, int32_t* new_of_old,
                      void* stream);

/* Copies the current CSR (device pointers): off has n_bfs+1 int64 entries,
 * col nnz int32 entries. Either may be NULL. Asynchronous. */
g3_status g3_get_csr(const g3_graph* g, int64_t* off, int32_t* col, void* stream);

/* Frees the graph and every device buffer it owns. It first waits for all
 * work on the current device (cudaDeviceSynchronize), so that the frees come
 * after any search still reading the graph on whatever stream it was queued.
 * NULL is a no-op. */
void g3_graph_free(g3_graph* g);

/* ---------------------------------------------------------------- BFS */

enum {
  G3_CTRL_HEURISTIC = 0, /* alpha/beta rule (Sec. 2.1, Beamer), on the device */
  G3_CTRL_LEARNED = 1,   /* 12-32-4 MLP on the device; paper has no counterpart */
  G3_CTRL_TOPDOWN = 2,   /* every level top-down (Algorithm 1/4) */
  G3_CTRL_BOTTOMUP = 3   /* every level after the first bottom-up (Algorithm 5) */
};

enum { G3_DIR_TD = 0, G3_DIR_BU = 1 };

typedef struct {
  int32_t controller;       /* G3_CTRL_* */
  int32_t alpha, beta;      /* heuristic: TD->BU when m_f*alpha > m_u; BU->TD when
                               the frontier shrank and n_f*beta < n_bfs (14, 24) */
  int32_t t1, t2, t3;       /* top-down degree bins: thread < t1 <= warp < t2 <=
                               CTA < t3 <= whole grid (32, 1024, 32768) */
  int32_t bu_reverse;       /* 1 (default): bottom-up scans each row from its
                               end (highest label first), Algorithm 6's
                               degree-aware order approximated under RCM;
                               0: CSR order as in Algorithm 5 */
  int32_t timing;           /* record per-level CUDA-event times in stats */
  const float* mlp_params;  /* device pointer, G3_MLP_NPARAMS floats, for
                               G3_CTRL_LEARNED */
  int32_t record_both;      /* training-data mode: every level is run both
                               top-down and bottom-up from the same state and
                               both are timed (stats t_td_ms, t_bu_ms) */
  int32_t mlp_margin;       /* learned controller: the network is evaluated
                               on the levels where the rule's own test is
                               within a factor of 4 of its threshold
                               (m_f*alpha against m_u, n_f*beta against
                               n_bfs) and overrides the rule's direction there
                               when its predicted |ln(t_BU / t_TD)| exceeds
                               mlp_margin / 1000 (0, the default: always) */
  int32_t mlp_bins;         /* learned controller: 1 (default) the network also
                               picks the top-down bins on the levels it is
                               evaluated on; 0 t1..t3 stay */
  int32_t out_split;        /* output pass (original IDs): 0 (default) and 1
                               one pass; 2 two passes over label halves (each
                               gathers from half of the packed (parent, level)
                               array) when both outputs are device memory */
  int32_t bu_kernel;        /* bottom-up kernels: 0 (default) word pairs -- a
                               lane owns one vertex of each of two bitmap words
                               -- on levels with at least a quarter of the
                               graph unvisited, and on the others a list of
                               the unvisited vertices with a thread for each
                               (Algorithm 6's shrinking active range); 1 with
                               bu_reverse, levels
                               with at least a quarter of the graph unvisited
                               run the staged kernel (each CTA's next tile of
                               neighbors+ entries and visited words brought into
                               shared memory by bulk copies while it works on
                               the current one) and the others the word-tile
                               kernel; without bu_reverse, word pairs; 2 word
                               tiles (a warp owns 32 words; dense tiles lane by
                               word, sparse ones as one compact list) on every
                               level; 3 word pairs on the levels with at least
                               a quarter of the graph unvisited, word tiles on
                               the others */
  int32_t stats_counts_only; /* 1: per-level statistics (stats, max_stats)
                               carry the counts but not the degree histogram
                               and label range (zero), so the expansion
                               kernels run as they do without statistics;
                               0 (default): everything */
  int32_t reserved[2];
} g3_bfs_opts;

/* Fills the defaults listed above. */
void g3_bfs_opts_default(g3_bfs_opts* o);

/* Statistics of one level: the frontier F_L expanded at that level. */
typedef struct {
  int32_t level;      /* L */
  int32_t dir;        /* G3_DIR_* used to expand F_L */
  int64_t n_f;        /* |F_L| */
  int64_t m_f;        /* sum of degrees over F_L */
  int64_t n_u;        /* vertices not in levels <= L */
  int64_t m_u;        /* sum of their degrees */
  int64_t examined;   /* bottom-up: edges examined (per unvisited vertex, up to
                         and including the first frontier neighbour); top-down:
                         m_f */
  int64_t n_next;     /* |F_{L+1}| */
  int32_t id_min, id_max; /* smallest / largest BFS-graph label in F_L */
  int64_t hist[4];    /* F_L vertices with degree in [0,32), [32,1024),
                         [1024,32768), [32768,inf) */
  int32_t t1, t2, t3; /* bin thresholds used (top-down levels) */
  float ms;           /* level time: format conversion, expansion and
                         controller kernels (opts.timing) */
  float ms_expand;    /* expansion kernels only: td_front..td_stats for a
                         top-down level, bu_pull for a bottom-up one */
  float t_td_ms, t_bu_ms; /* record_both: best top-down time over the
                             threshold candidates, bottom-up time */
  int32_t best_t1, best_t2, best_t3; /* record_both: fastest top-down bins */
  float mlp_out[4];   /* learned controller outputs for this level */
} g3_level_stats;

/* Breadth-first search from `root` (original ID) on the graph's current CSR
 * (Algorithm 2): each level expanded top-down from a frontier queue
 * (degree-binned thread / warp / CTA / grid work, Algorithms 1 and 4) or
 * bottom-up over the unvisited vertices with bitmaps and an early exit on
 * the first parent found (Algorithm 5; on levels with under 4 % of the graph
 * unvisited, over a list of those vertices, Algorithm 6's shrinking active
 * range), as the controller decides. After a full RCM relabel the output
 * pass takes the reached set from the root's component range.
 *   parent, level : n int32 entries each (original IDs); device OR host
 *                   pointers. Page-locked host memory is written directly
 *                   by the output kernel; pageable host memory is filled
 *                   through a device staging copy.
 *                   parent[root] = root, level[root] = 0; unreachable and
 *                   isolated vertices get -1 in both. An isolated root is
 *                   valid: only the root is reached.
 *   opts          : NULL = defaults.
 *   stats         : host array of max_stats entries or NULL; receives one
 *                   record per level while room remains (degree histogram
 *                   and label range included unless opts.stats_counts_only). *n_levels (may be
 *                   NULL) receives the number of non-empty frontiers.
 * The first call on a graph allocates its BFS workspace (about 52 bytes per
 * BFS vertex plus 8 per vertex of the input); later calls allocate nothing. By default the level loop runs on
 * the device as one CUDA graph (a WHILE node over a SWITCH of level kinds,
 * conditions set by the device-side controller; rebuilt when the options
 * change) and the call synchronises `stream` once after it and before
 * returning. With opts.timing or opts.record_both the loop is driven from the
 * host instead and synchronises once per level (the controller's record is
 * read back). Searches deeper than 4096 levels continue on the host loop.
 * Errors: G3_EINVAL (root outside [0, n), null parent/level, learned
 * controller without parameters), G3_ENOMEM, G3_ECUDA, G3_ETIMEOUT (a
 * kernel's bounded wait for its staged data ran out; the search stopped and
 * the outputs are not valid). */
g3_status g3_bfs(g3_graph* g, int32_t root, const g3_bfs_opts* opts, int32_t* parent,
                 int32_t* level, g3_level_stats* stats, int32_t max_stats,
                 int32_t* n_levels, void* stream);

/* --------------------------------------------------- multi-source BFS */

/* Up to 64 searches in one pass, one bit per source in a uint64 per vertex
 * (the paper runs its 64 evaluation roots one after the other, Sec. 4; this
 * batched form has no counterpart there). Per level the frontier is either
 * pushed (every frontier vertex ORs its source bits into its neighbours,
 * the top-down analogue of Algorithm 1) or pulled (every vertex not reached
 * by all sources ORs its neighbours' frontier words, with an early exit once
 * all missing sources are found, the bottom-up analogue of Algorithm 2). */
typedef struct {
  int32_t push_alpha;     /* pull a level when (sum of frontier degrees) *
                             push_alpha > nnz, else push (14) */
  int32_t pull_warp_deg;  /* pull: vertices of at least this degree are scanned
                             by a whole warp, smaller ones by one thread (256) */
  int32_t reserved[6];
} g3_msbfs_opts;

void g3_msbfs_opts_default(g3_msbfs_opts* o);

/* BFS from roots[0..k) (host array, original IDs, 1 <= k <= 64; repeats
 * allowed) on the graph's current CSR.
 *   level    : device pointer, k x n int8, row s = hop distances from roots[s]
 *              in original IDs, -1 where unreachable (isolated roots reach
 *              only themselves).
 *   n_levels : (nullable) number of levels run.
 *   ms       : (nullable) time of the call on the device, CUDA events.
 * The first call on a graph allocates its workspace (about 112 bytes per
 * BFS vertex). The level loop runs on the device as one CUDA graph (a WHILE
 * node over a push/pull SWITCH, decided by a device-side control kernel;
 * rebuilt when k's source mask or the options change); the call synchronises
 * `stream` once, before returning.
 * Errors: G3_EINVAL, G3_ERANGE (a level above 126 does not fit int8),
 * G3_ENOMEM, G3_ECUDA. */
g3_status g3_msbfs(g3_graph* g, const int32_t* roots, int32_t k, const g3_msbfs_opts* opts,
                   int8_t* level, int32_t* n_levels, float* ms, void* stream);

/* Work counts of the last g3_msbfs call on the graph (for the roofline). */
typedef struct {
  int32_t levels, pull_levels, push_levels, reserved;
  int64_t pull_entries;   /* row entries the pull levels read (early exits counted
                             where they happened) */
  int64_t pull_vertices;  /* vertices whose rows the pull levels scanned */
  int64_t push_entries;   /* row entries of the pushed frontier vertices */
} g3_msbfs_stats;

/* Copies the counts of the last g3_msbfs call. Host only, no synchronisation.
 * Errors: G3_EINVAL, G3_ESTATE (no multi-source search on the graph yet). */
g3_status g3_msbfs_last_stats(const g3_graph* g, g3_msbfs_stats* out);

/* ------------------------------------------------- batched small graphs */

/* Many small graphs searched in one persistent, CUDA-graph-captured launch
 * (no counterpart in the paper). */
typedef struct g3_batch g3_batch;

typedef struct {
  int32_t warp_max_n;  /* mode 0: graphs with at most this many BFS vertices are
                          searched by one warp, larger ones by a whole CTA (1024;
                          at most 2048 are ever given to a warp) */
  int32_t mode;        /* 0 (default): one persistent kernel, each graph searched
                          by its own warp or CTA with its bitmaps in shared
                          memory, captured once into a CUDA graph; 1: one
                          level-synchronous search over the union of the graphs
                          seeded with all roots at once (the graphs are disjoint,
                          so the levels of one cannot reach another), run by the
                          single-source kernels and level-loop graph */
  int32_t reserved[6];
} g3_batch_opts;

void g3_batch_opts_default(g3_batch_opts* o);

/* Packs G graphs, each built by g3_build_csr and relabelled by g3_rcm_relabel,
 * into one union: graph g keeps the contiguous ID range [voff[g], voff[g+1])
 * (voff = prefix sums of the graphs' n in the given order) for original IDs and
 * labels alike. The graphs are read, not taken over: the caller may free them
 * afterwards. Each graph may have at most 16384 non-isolated vertices.
 * Synchronises. Errors: G3_EINVAL, G3_ENOMEM, G3_ECUDA. */
g3_status g3_batch_pack(g3_graph* const* graphs, int32_t G, void* stream, g3_batch** out);

g3_status g3_batch_info_get(const g3_batch* b, int32_t* G, int64_t* N, int64_t* nnz);

/* One BFS per graph: roots (device, G entries, union original IDs, root g in
 * graph g's range), parent and level (device, N entries each, union original
 * IDs; a root outside its graph's range leaves that graph all -1). Mode 0: the
 * first call with a given (roots, parent, level, warp_max_n) captures the
 * launch into a CUDA graph, later calls only launch it; asynchronous unless ms
 * is given. Mode 1: synchronises (the controller's record is read back).
 * ms (nullable): device time of the call, which then synchronises. */
g3_status g3_bfs_batch(g3_batch* b, const int32_t* roots, const g3_batch_opts* opts,
                       int32_t* parent, int32_t* level, float* ms, void* stream);

void g3_batch_free(g3_batch* b);

/* ------------------------------------------------------------ autotuner */

/* Device-timed search over launch parameters with a per-size-class cache
 * file. The paper picks its switching parameters by a grid search over
 * measured runs (Sec. 4); these calls extend that search to the parameters
 * of this library's kernels. Each candidate is timed as the minimum of three
 * runs, each after a 256 MB write that evicts L2. */
enum { G3_TUNE_BFS = 1, G3_TUNE_MSBFS = 2, G3_TUNE_BATCH = 3 };

typedef struct {
  int32_t kind;        /* G3_TUNE_* */
  int32_t size_class;  /* floor(log2(BFS vertices per graph)) */
  int32_t deg_class;   /* floor(log2(CSR entries per BFS vertex)) */
  int32_t p[6];        /* chosen values: BFS (alpha, beta, t1, t2, t3, bu_reverse);
                          MS-BFS (push_alpha, pull_warp_deg); batch (warp_max_n,
                          mode);
                          unused slots 0 */
  int32_t points;      /* candidates timed; 0 when the entry came from the cache */
  float ms;            /* device ms of the chosen point (BFS: summed over roots) */
  float ms_default;    /* device ms of the options passed in */
} g3_tune_entry;

/* Size class of a graph (graphs = 1) or of a batch (graphs = G, vertices and
 * nnz the batch totals). Host only. Errors: G3_EINVAL. */
g3_status g3_tune_key(int32_t kind, int64_t vertices, int64_t nnz, int32_t graphs,
                      int32_t* size_class, int32_t* deg_class);

/* Cache file access, host only. A missing or unreadable file holds no entries
 * (lookup sets *found = 0); malformed lines are skipped; the last line with a
 * key wins. Store rewrites the file (through path.tmp and a rename) with the
 * entry replacing any of the same key. Errors: G3_EINVAL (null argument, bad
 * kind, file not writable). */
g3_status g3_tune_cache_lookup(const char* path, int32_t kind, int32_t size_class,
                               int32_t deg_class, g3_tune_entry* out, int32_t* found);
g3_status g3_tune_cache_store(const char* path, const g3_tune_entry* e);

/* Each autotune call first looks up its key in cache_path (nullable: no
 * cache) and, on a hit, only copies the cached values into *opts. Otherwise it
 * times the candidates on the device, writes the fastest into *opts (which
 * on entry holds the starting point and every option not searched), stores it
 * in the cache and fills *rec (nullable). Outputs of the timed runs are left
 * in the caller's buffers. Synchronises.
 *   g3_autotune_bfs   : roots host (nroots original IDs), parent/level as for
 *                       g3_bfs; coordinate search, two passes, over alpha,
 *                       beta, (t1, t2, t3), bu_reverse and bu_kernel (0, 1 or 3);
 *                       the controller stays.
 *   g3_autotune_msbfs : roots host (k <= 64), level as for g3_msbfs; full grid
 *                       over push_alpha x pull_warp_deg.
 *   g3_autotune_batch : roots/parent/level as for g3_bfs_batch; mode 0 with
 *                       warp_max_n over {0, 64, ..., 2048}, and mode 1.
 * Errors: those of the timed call, G3_EINVAL, G3_ENOMEM. */
g3_status g3_autotune_bfs(g3_graph* g, const int32_t* roots, int32_t nroots, int32_t* parent,
                          int32_t* level, const char* cache_path, g3_bfs_opts* opts,
                          g3_tune_entry* rec, void* stream);
g3_status g3_autotune_msbfs(g3_graph* g, const int32_t* roots, int32_t k, int8_t* level,
                            const char* cache_path, g3_msbfs_opts* opts, g3_tune_entry* rec,
                            void* stream);
g3_status g3_autotune_batch(g3_batch* b, const int32_t* roots, int32_t* parent, int32_t* level,
                            const char* cache_path, g3_batch_opts* opts, g3_tune_entry* rec,
                            void* stream);

/* --------------------------------------------------- learned controller */

/* The learned direction / binning controller (the paper has no learned
 * part; it tunes alpha and beta by grid search, Sec. 3.6): a multilayer
 * perceptron with 12 inputs, 32 ReLU hidden units and 4 linear outputs.
 *   params : G3_MLP_NPARAMS floats, layout W1[32][12], b1[32], W2[4][32], b2[4]
 *   x      : B rows of 12 features (see g3_mlp_features), row-major
 *   y      : B rows of 4 targets: ln(t_BU / t_TD) and log2 of the fastest
 *            top-down bin thresholds t1, t2, t3
 *   w      : 4 per-output loss weights, or NULL for all ones
 * Loss L = 1/(2B) sum_b sum_k w_k (o_bk - y_bk)^2. All pointers are device
 * pointers; calls are asynchronous on `stream` unless stated. */
#define G3_MLP_NPARAMS 548

/* out: B rows of 4 outputs. o0 < 0 selects bottom-up. */
g3_status g3_mlp_forward(const float* params, const float* x, int32_t B, float* out,
                         void* stream);

/* loss (1 float) and grad (G3_MLP_NPARAMS floats) of the batch; computed by
 * one block with a fixed summation order, so repeated calls agree bit for bit. */
g3_status g3_mlp_loss_grad(const float* params, const float* x, const float* y,
                           const float* w, int32_t B, float* loss, float* grad,
                           void* stream);

/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) at rate lr,
 * updating params in place; losses (steps floats, or NULL) receives the loss
 * before each step. One kernel launch. */
g3_status g3_mlp_train(float* params, const float* x, const float* y, const float* w,
                       int32_t B, int32_t steps, float lr, float* losses, void* stream);

/* Feature rows x (count x 12 floats, device) of the level records `stats`
 * (host array as g3_bfs returns them, consecutive records of one search in
 * order), computed by the same device code the controller uses. n_bfs and
 * nnz are the searched graph's vertex and directed-entry counts (the
 * features are ratios to them). Synchronises `stream`. */
g3_status g3_mlp_features(const g3_level_stats* stats, int32_t count, int32_t n_bfs, int64_t nnz,
                          float* x, void* stream);

/* ------------------------------------------------------ test hooks */

/* Fault injection for tests of the error paths (the paper has no
 * counterpart). G3_INJECT_ALLOC: the value-th device allocation the library
 * makes from now on (every stream-ordered buffer and every workspace buffer
 * of any call) fails as if the device were out of memory, once; the call
 * then returns G3_ENOMEM with nothing of its own left allocated and the
 * graph as it was before the call. value <= 0 disarms it.
 * G3_INJECT_RCM_ROUNDS: caps the rounds of component hooking in the RCM
 * relabel (default 4096); a relabel that needs more returns G3_ETIMEOUT and
 * leaves the graph not relabelled. value <= 0 restores the default.
 * G3_INJECT_STAGED_STALL: the staged bottom-up kernel (bu_kernel 1) leaves
 * out the bulk copies of each CTA's first tile and polls that tile's barrier
 * only `value` times, so its bounded wait runs out: the search stops and
 * g3_bfs returns G3_ETIMEOUT, with the device left usable. value <= 0 turns
 * it off (the wait limit returns to its default).
 * Process-wide; not for concurrent use. Errors: G3_EINVAL (unknown kind),
 * G3_ECUDA. */
enum { G3_INJECT_ALLOC = 1, G3_INJECT_RCM_ROUNDS = 2, G3_INJECT_STAGED_STALL = 3 };
g3_status g3_debug_inject(int32_t kind, int64_t value);

/* Bytes currently allocated from the current device's default memory pool
 * (the pool the stream-ordered buffers come from), for leak checks around a
 * failed call. Errors: G3_EINVAL (null), G3_ECUDA. */
g3_status g3_debug_pool_used(int64_t* bytes);

/* ------------------------------------------------- allocation-free BFS */

/* The paper has no counterpart to this entry point: it serves callers that
 * cannot allocate device memory when they search -- code running inside a
 * host framework that has already reserved the device memory for its own
 * pool, or latency-critical paths where cudaMalloc / cudaFree could
 * synchronise the device. It performs a level-synchronous top-down BFS over
 * a caller-provided CSR and allocates nothing: its scratch (visited bitmap,
 * two frontier queues, counters) is one fixed-size static device array of
 * 8,519,936 bytes (about 8.5 MB) that every GPU loading the library holds
 * until the process exits.
 *   off, col      : device pointers, CSR of an undirected graph with n rows
 *                   (off: n+1 int64, col: off[n] int32 entries, as produced by
 *                   g3_get_csr), read only.
 *   n             : 1 <= n <= G3_NOALLOC_MAX_N; larger n is rejected with
 *                   G3_EINVAL before anything runs.
 *   root          : in [0, n).
 *   parent, level : device pointers, n int32 entries each, in the CSR's own
 *                   vertex IDs (no relabelling); -1 for unreachable vertices.
 * All calls on a device share the scratch array, which keeps the last call's
 * contents (each call clears what must start at zero): calls whose GPU work
 * overlaps race, so serialise them. The first call on a device looks up the
 * array's address (cudaGetSymbolAddress, that device current); make that
 * first call before any stream capture. The address is cached per device for
 * the life of the process: after cudaDeviceReset on that device, do not call
 * this entry point again. Synchronises `stream` once per level.
 * Errors: G3_EINVAL, G3_ECUDA. */
#define G3_NOALLOC_MAX_N (1 << 20)
g3_status g3_bfs_noalloc(const int64_t* off, const int32_t* col, int32_t n, int32_t root,
                         int32_t* parent, int32_t* level, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* G3BFS_H */
