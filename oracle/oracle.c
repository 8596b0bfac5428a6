/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, serial and obviously correct restatement of what the BFS/RCM
 * path computes (Jiang et al., "Fast and Efficient Parallel Breadth-First
 * Search with Power-law Graph Transformation", PPoPP'21). It is used only by
 * the tests, by the package's smoke check and by the benchmark's CPU-baseline
 * leg; the product path never calls it. It shares no code with the CUDA
 * library: no headers, helpers or tables.
 *
 * Functions and the passages they follow:
 *   orc_build_csr     Sec. 3.1 / Eq. 2: undirected graph stored as CSR
 *                     (row_starts, dst), both directions; self-loops and
 *                     duplicate tuples of the generated edge list removed
 *                     (Sec. 4.2 notes the generator produces both).
 *   orc_rcm           Algorithm 3 (Reverse Cuthill-McKee) step by step:
 *                     V+ by increasing degree, sorted_neighbors by increasing
 *                     degree, start of each component = first unvisited
 *                     vertex of V+ (minimal degree, Sec. 3.2), FIFO relabel,
 *                     reverse, append V \ V+.
 *   orc_rcm_partial   partial RCM (Sec. 4.6): Algorithm 3 on the top p of
 *                     V+ only, the rest in ID order (reading in its comment).
 *   orc_rcm_check     certificate check that a permutation is Algorithm 3's
 *                     output (the conditions that make it unique), for sizes
 *                     where running Algorithm 3 itself takes too long.
 *   orc_permute_csr   the relabelled CSR the BFS runs on (isolated vertices
 *                     dropped, Sec. 1 contribution 1; rows ascending).
 *   orc_bfs           Algorithm 1 run serially: FIFO frontier, neighbours in
 *                     CSR order, the first discoverer becomes the predecessor;
 *                     pi(s)=s, -1 when unreachable (Sec. 2.1).
 *   orc_validate      the predecessor-map rules implied by Sec. 2.1;
 *                     orc_validate_tree the same rules but the edge pass,
 *                     for levels already compared with orc_bfs.
 *   orc_bandwidth     Eq. 1.
 *   orc_bu_examined   edges a bottom-up step examines (Algorithm 2, bottom-up
 *                     branch): per unvisited vertex, neighbours in CSR order up
 *                     to and including the first one in the current frontier.
 *
 * Readings of points the paper leaves open:
 *   - degree = number of distinct neighbours other than the vertex itself,
 *     i.e. the row length of the cleaned CSR;
 *   - ties in "increasing order of degree" (Algorithm 3) are broken by
 *     ascending original vertex ID;
 *   - P is the array position -> original ID; after reversal the vertex at
 *     position i of P gets new label i;
 *   - isolated vertices V \ V+ are appended in ascending original ID.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ CSR */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Builds the cleaned CSR of the undirected graph given by m tuples.
 * off: n+1 entries; col: capacity 2*m. Returns nnz (directed entries). */
int64_t orc_build_csr(const int32_t* src, const int32_t* dst, int64_t m,
                      int32_t n, int64_t* off, int32_t* col) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i) {
    if (src[i] == dst[i]) continue;            /* self-loop dropped */
    cnt[src[i]]++;
    cnt[dst[i]]++;                             /* stored in both directions */
  }
  int64_t* pos = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  pos[0] = 0;
  for (int32_t v = 0; v < n; ++v) pos[v + 1] = pos[v] + cnt[v];
  int64_t* fill = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  memcpy(fill, pos, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v) continue;
    col[fill[u]++] = v;
    col[fill[v]++] = u;
  }
  /* sort each row ascending and drop duplicate neighbours */
  int64_t w = 0;
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) {
    int64_t b = pos[v], e = pos[v + 1];
    qsort(col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
    for (int64_t i = b; i < e; ++i)
      if (i == b || col[i] != col[i - 1]) col[w++] = col[i];
    off[v + 1] = w;
  }
  free(cnt);
  free(pos);
  free(fill);
  return w;
}

/* ------------------------------------------------------------------ RCM */

static _Thread_local const int64_t* g_off;

static int64_t deg_of(int32_t v) { return g_off[v + 1] - g_off[v]; }

/* increasing degree, ties by ascending ID */
static int cmp_deg_id(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  int64_t dx = deg_of(x), dy = deg_of(y);
  if (dx != dy) return (dx > dy) - (dx < dy);
  return (x > y) - (x < y);
}

/* Algorithm 3. P (n entries) receives the permutation, position -> original
 * ID: positions [0, |V+|) hold the reversed Cuthill-McKee order, positions
 * [|V+|, n) the isolated vertices. Returns |V+|. */
int32_t orc_rcm(const int64_t* off, const int32_t* col, int32_t n, int32_t* P) {
  g_off = off;
  /* V+ : non-isolated vertices in increasing order of degree */
  int32_t* vplus = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t np = 0;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) > 0) vplus[np++] = v;
  qsort(vplus, (size_t)np, sizeof(int32_t), cmp_deg_id);

  uint8_t* visited = (uint8_t*)calloc((size_t)n + 1, 1);
  int64_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) > maxdeg) maxdeg = deg_of(v);
  int32_t* nb = (int32_t*)malloc(((size_t)maxdeg + 1) * sizeof(int32_t));

  int32_t min_index = 0, slow = 0, fast = 0;
  while (slow < np) {
    /* next unvisited vertex with the minimal degree starts a component */
    for (int32_t i = min_index; i < np; ++i) {
      if (!visited[vplus[i]]) {
        P[slow] = vplus[i];
        visited[vplus[i]] = 1;
        min_index = i + 1;
        fast = slow + 1;
        break;
      }
    }
    /* explore the component, relabelling unvisited neighbours in
     * increasing order of degree */
    while (slow < fast) {
      int32_t v = P[slow];
      int64_t d = deg_of(v);
      memcpy(nb, col + off[v], (size_t)d * sizeof(int32_t));
      qsort(nb, (size_t)d, sizeof(int32_t), cmp_deg_id); /* sorted_neighbors(v) */
      for (int64_t j = 0; j < d; ++j) {
        int32_t w = nb[j];
        if (!visited[w]) {
          visited[w] = 1;
          P[fast++] = w;
        }
      }
      slow++;
    }
  }
  /* P = reverse(P) */
  for (int32_t i = 0, j = np - 1; i < j; ++i, --j) {
    int32_t t = P[i]; P[i] = P[j]; P[j] = t;
  }
  /* P.append(V \ V+) */
  int32_t k = np;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) == 0) P[k++] = v;
  free(vplus);
  free(visited);
  free(nb);
  return np;
}

/* Partial RCM (Sec. 4.6): only the top p of V+ is reordered. The paper gives
 * no procedure; the reading taken here: the top k = ceil(p_permille * |V+| /
 * 1000) vertices are the last k of V+ in Algorithm 3's (degree, ID) order.
 * Algorithm 3 runs on that set S alone (starts and neighbour orders as in
 * orc_rcm, with the graph's degrees; neighbours outside S ignored), and its
 * reversed order fills positions 0..k-1. The rest of V+ follows in ascending
 * original ID, then V \ V+. p_permille = 1000 gives orc_rcm exactly.
 * Returns n_plus. */
int32_t orc_rcm_partial(const int64_t* off, const int32_t* col, int32_t n,
                        int32_t p_permille, int32_t* P) {
  g_off = off;
  int32_t* vplus = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t np = 0;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) > 0) vplus[np++] = v;
  qsort(vplus, (size_t)np, sizeof(int32_t), cmp_deg_id);
  if (p_permille < 0) p_permille = 0;
  if (p_permille > 1000) p_permille = 1000;
  const int32_t k = (int32_t)(((int64_t)np * p_permille + 999) / 1000);
  const int32_t lo = np - k; /* S = vplus[lo .. np) */

  uint8_t* in_s = (uint8_t*)calloc((size_t)n + 1, 1);
  for (int32_t i = lo; i < np; ++i) in_s[vplus[i]] = 1;
  uint8_t* visited = (uint8_t*)calloc((size_t)n + 1, 1);
  int64_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) > maxdeg) maxdeg = deg_of(v);
  int32_t* nb = (int32_t*)malloc(((size_t)maxdeg + 1) * sizeof(int32_t));

  int32_t min_index = lo, slow = 0, fast = 0;
  while (slow < k) {
    for (int32_t i = min_index; i < np; ++i) {
      if (!visited[vplus[i]]) {
        P[slow] = vplus[i];
        visited[vplus[i]] = 1;
        min_index = i + 1;
        fast = slow + 1;
        break;
      }
    }
    while (slow < fast) {
      int32_t v = P[slow];
      int64_t d = deg_of(v);
      memcpy(nb, col + off[v], (size_t)d * sizeof(int32_t));
      qsort(nb, (size_t)d, sizeof(int32_t), cmp_deg_id);
      for (int64_t j = 0; j < d; ++j) {
        int32_t w = nb[j];
        if (in_s[w] && !visited[w]) {
          visited[w] = 1;
          P[fast++] = w;
        }
      }
      slow++;
    }
  }
  for (int32_t i = 0, j = k - 1; i < j; ++i, --j) {
    int32_t t = P[i]; P[i] = P[j]; P[j] = t;
  }
  int32_t q = k;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) > 0 && !in_s[v]) P[q++] = v;
  for (int32_t v = 0; v < n; ++v)
    if (deg_of(v) == 0) P[q++] = v;
  free(vplus);
  free(in_s);
  free(visited);
  free(nb);
  return np;
}

/* Certificate check of an RCM permutation against Algorithm 3, without
 * running Algorithm 3 (whose per-row sorts take many minutes at 2^26
 * vertices). P maps position -> original ID as orc_rcm returns it. Let Q be
 * the Cuthill-McKee order (P[0 .. n_plus) read backwards), pos[v] the
 * position of v in Q, and mp(w) / mx(w) the smallest / largest position of a
 * neighbour of w. Algorithm 3 appends a vertex either as the start of a new
 * component (its queue being empty) or while dequeuing its earliest-placed
 * neighbour, the unvisited neighbours of each dequeued vertex in increasing
 * (degree, ID). Its Q is therefore the one order of V+ with
 *   1. P a permutation of [0, n); P[0 .. n_plus) = V+ (degree > 0) and
 *      P[n_plus .. n) = V \ V+ in ascending ID;
 *   2. a vertex with mp(w) > pos(w) (a start) comes when every vertex before
 *      it has all its neighbours before it (the queue is empty), and it is
 *      the minimal (degree, ID) vertex among Q[pos(w) ..];
 *   3. the other vertices (mp(w) < pos(w)) appear in strictly increasing
 *      (mp(w), degree(w), ID(w)).
 * Uniqueness: if Q' satisfies 1-3 and first differs from Algorithm 3's Q at
 * position j, then either Q[j] is a start, whose queue-empty state and
 * minimality rule 2 gives to Q'[j] as well, or Q[j] has a neighbour in the
 * common prefix, so Q'[j] cannot be a start (rule 2) and rule 3 orders Q[j]
 * before Q'[j] by the same key in both orders -- a contradiction either way.
 * Returns 0 when P passes, else the rule number with the offending position
 * in *bad. */
int32_t orc_rcm_check(const int64_t* off, const int32_t* col, int32_t n,
                      const int32_t* P, int64_t* bad) {
  *bad = -1;
  int32_t np = 0;
  for (int32_t v = 0; v < n; ++v)
    if (off[v + 1] > off[v]) np++;
  int32_t* pos = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  uint8_t* start = (uint8_t*)calloc((size_t)n + 1, 1);
  for (int32_t v = 0; v < n; ++v) pos[v] = -1;
  int32_t rc = 0;
  /* rule 1 */
  for (int32_t i = 0; i < n && !rc; ++i) {
    int32_t v = P[i];
    if (v < 0 || v >= n || pos[v] >= 0) { rc = 1; *bad = i; break; }
    int64_t d = off[v + 1] - off[v];
    if ((i < np) != (d > 0)) { rc = 1; *bad = i; break; }
    if (i > np && P[i] < P[i - 1]) { rc = 1; *bad = i; break; }
    pos[v] = i < np ? np - 1 - i : i; /* Cuthill-McKee position */
  }
  /* forward pass: rules 2 (queue empty) and 3 */
  int64_t prefmax = -1;
  int64_t k_mp = -1, k_deg = -1, k_id = -1; /* key of the last non-start */
  for (int32_t j = 0; j < np && !rc; ++j) {
    int32_t w = P[np - 1 - j];
    int64_t mp = INT64_MAX, mx = -1;
    for (int64_t e = off[w]; e < off[w + 1]; ++e) {
      int64_t q = pos[col[e]];
      if (q < mp) mp = q;
      if (q > mx) mx = q;
    }
    int64_t d = off[w + 1] - off[w];
    if (mp > j) { /* a start: no vertex before it has a neighbour after it */
      start[j] = 1;
      if (prefmax >= j) { rc = 2; *bad = j; break; }
    } else {
      if (mp < k_mp || (mp == k_mp && (d < k_deg || (d == k_deg && w <= k_id)))) {
        rc = 3;
        *bad = j;
        break;
      }
      k_mp = mp;
      k_deg = d;
      k_id = w;
    }
    if (mx > prefmax) prefmax = mx;
  }
  /* backward pass: rule 2 (a start is the minimal (degree, ID) remaining) */
  int64_t b_deg = INT64_MAX, b_id = INT64_MAX;
  for (int32_t j = np - 1; j >= 0 && !rc; --j) {
    int32_t w = P[np - 1 - j];
    int64_t d = off[w + 1] - off[w];
    if (d < b_deg || (d == b_deg && w < b_id)) {
      b_deg = d;
      b_id = w;
    }
    if (start[j] && b_id != w) { rc = 2; *bad = j; }
  }
  free(pos);
  free(start);
  return rc;
}

/* Relabelled CSR over the n_plus non-isolated vertices: row i holds the new
 * labels of the neighbours of original vertex P[i], ascending.
 * off_new: n_plus+1 entries; col_new: nnz entries. */
void orc_permute_csr(const int64_t* off, const int32_t* col, int32_t n,
                     const int32_t* P, int32_t n_plus, int64_t* off_new,
                     int32_t* col_new) {
  int32_t* label = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) label[P[i]] = i;
  off_new[0] = 0;
  for (int32_t i = 0; i < n_plus; ++i) {
    int32_t v = P[i];
    int64_t b = off_new[i];
    for (int64_t j = off[v]; j < off[v + 1]; ++j) col_new[b + (j - off[v])] = label[col[j]];
    int64_t d = off[v + 1] - off[v];
    qsort(col_new + b, (size_t)d, sizeof(int32_t), cmp_i32);
    off_new[i + 1] = b + d;
  }
  free(label);
}

/* ------------------------------------------------------------------ BFS */

/* Serial level-synchronous BFS (Algorithm 1 with one thread). parent and
 * level have n entries; -1 marks unreachable vertices. */
void orc_bfs(const int64_t* off, const int32_t* col, int32_t n, int32_t root,
             int32_t* parent, int32_t* level) {
  for (int32_t v = 0; v < n; ++v) { parent[v] = -1; level[v] = -1; }
  if (root < 0 || root >= n) return;
  int32_t* queue = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int64_t head = 0, tail = 0;
  parent[root] = root;
  level[root] = 0;
  queue[tail++] = root;
  while (head < tail) {
    int32_t v = queue[head++];
    for (int64_t j = off[v]; j < off[v + 1]; ++j) {
      int32_t w = col[j];
      if (level[w] < 0) {
        level[w] = level[v] + 1;
        parent[w] = v;
        queue[tail++] = w;
      }
    }
  }
  free(queue);
}

static int has_edge(const int64_t* off, const int32_t* col, int32_t u, int32_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) { /* rows are ascending */
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == v) return 1;
    if (col[mid] < v) lo = mid + 1; else hi = mid;
  }
  return 0;
}

/* Checks a (parent, level) pair for root against the graph.
 * Returns 0 when valid, else the number of the first rule broken, with the
 * offending vertex in *bad:
 *   1  parent[root] == root and level[root] == 0
 *   2  every other reached v: (parent[v], v) is an edge and
 *      level[v] == level[parent[v]] + 1
 *   3  the root is the only vertex at level 0 (so every parent chain ends at
 *      the root and, with rule 5, the reached set is the root's component)
 *   4  parent[v] == -1 exactly when level[v] == -1
 *   5  every edge joins two unreached vertices or two reached vertices whose
 *      levels differ by at most one
 * Rules 2 and 5 together force level[] to equal the hop distance. */
static int32_t validate_tree_rules(const int64_t* off, const int32_t* col, int32_t n,
                                   int32_t root, const int32_t* parent,
                                   const int32_t* level, int64_t* bad) {
  *bad = -1;
  if (root < 0 || root >= n || parent[root] != root || level[root] != 0) {
    *bad = root;
    return 1;
  }
  for (int32_t v = 0; v < n; ++v) {
    if ((parent[v] == -1) != (level[v] == -1)) { *bad = v; return 4; }
  }
  for (int32_t v = 0; v < n; ++v) {
    if (level[v] == 0 && v != root) { *bad = v; return 3; }
    if (v == root || parent[v] == -1) continue;
    int32_t p = parent[v];
    if (p < 0 || p >= n || p == v || level[p] < 0 || level[v] != level[p] + 1 ||
        !has_edge(off, col, p, v)) {
      *bad = v;
      return 2;
    }
  }
  return 0;
}

int32_t orc_validate(const int64_t* off, const int32_t* col, int32_t n,
                     int32_t root, const int32_t* parent, const int32_t* level,
                     int64_t* bad) {
  int32_t r = validate_tree_rules(off, col, n, root, parent, level, bad);
  if (r) return r;
  for (int32_t u = 0; u < n; ++u) {
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      int32_t w = col[j];
      int ru = level[u] >= 0, rw = level[w] >= 0;
      if (ru != rw) { *bad = u; return 5; }
      if (ru && (level[u] - level[w] > 1 || level[w] - level[u] > 1)) { *bad = u; return 5; }
    }
  }
  return 0;
}

/* Rules 1-4 of orc_validate only, for a level[] already known to equal the
 * hop distances (compared with orc_bfs), where rule 5 holds by itself: the
 * parents then form a BFS tree exactly when rules 1-4 hold. Skips the pass
 * over every edge, which dominates orc_validate on large graphs. */
int32_t orc_validate_tree(const int64_t* off, const int32_t* col, int32_t n,
                          int32_t root, const int32_t* parent, const int32_t* level,
                          int64_t* bad) {
  return validate_tree_rules(off, col, n, root, parent, level, bad);
}

/* Eq. 1: BW(A) = max{ i - j : A_ij != 0, i > j } under the labelling
 * label[v] (identity when label is NULL). */
int64_t orc_bandwidth(const int64_t* off, const int32_t* col, int32_t n,
                      const int32_t* label) {
  int64_t bw = 0;
  for (int32_t u = 0; u < n; ++u) {
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      int64_t a = label ? label[u] : u, b = label ? label[col[j]] : col[j];
      if (a - b > bw) bw = a - b;
    }
  }
  return bw;
}

/* Edges examined by the bottom-up step from level L to L+1 (Algorithm 2,
 * bottom-up branch, with the early break): for each vertex not yet visited
 * (level > L or -1), its neighbours in CSR order up to and including the
 * first one at level L, or all of them when there is none. With reverse != 0
 * rows are scanned from their end (highest label first). */
int64_t orc_bu_examined(const int64_t* off, const int32_t* col, int32_t n,
                        const int32_t* level, int32_t L, int32_t reverse) {
  int64_t total = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (level[v] >= 0 && level[v] <= L) continue;
    int64_t d = off[v + 1] - off[v], k = 0;
    for (; k < d; ++k) {
      int32_t w = reverse ? col[off[v + 1] - 1 - k] : col[off[v] + k];
      if (level[w] == L) { k++; break; }
    }
    total += k;
  }
  return total;
}
