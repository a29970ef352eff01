/*
 * CPU oracle for the minimum spanning forest (MSF).  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * GPU solver never calls, links or includes it, and it shares no code with it.
 *
 * Problem (paper Section 2.2, "Graph and Input/Output Format"): an undirected
 * weighted graph G = (V, E); the output is a minimum spanning tree of every
 * connected component, i.e. a minimum spanning forest.  Vertices are 0-based
 * here (the paper numbers them 1..|V|).
 *
 * Order (Section 2.3: ties are broken consistently so that edge weights can be
 * assumed distinct and the MST is unique): edge e precedes edge f iff
 * (w_e, id_e) < (w_f, id_f) lexicographically, id = position in the input.
 * Under this strict total order the MSF is unique; every function below returns
 * that forest as ascending edge ids plus its total weight as a uint64.
 * Self-loops are never forest edges; parallel edges are allowed.
 *
 * Functions:
 *   oracle_kruskal   Kruskal: edges in (w,id) order, union-find, keep an edge
 *                    iff it joins two different trees.
 *   oracle_kruskal_par  The same Kruskal with its sort spread over host
 *                    threads (each radix pass: per-thread digit counts over
 *                    contiguous chunks, then a stable scatter); the
 *                    union-find pass stays sequential.  For timing on many
 *                    cores; its output equals oracle_kruskal's.
 *   oracle_prim      Jarnik-Prim with a binary heap keyed by (w,id), restarted
 *                    from every unvisited vertex (an independent cross-check).
 *   oracle_brute     Exhaustive search over edge subsets for tiny graphs.
 *   oracle_check_msf Spanning-forest, cut-property and cycle-property checks.
 * Status codes: 0 ok, 1 vertex id out of range, 2 graph too large for the
 * routine, 3 out of memory.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KEY(w, id) ((((uint64_t)(w)) << 32) | (uint64_t)(id))

static int check_range(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst) {
  for (uint64_t e = 0; e < m; ++e)
    if (src[e] >= n || dst[e] >= n) return 1;
  return 0;
}

/* ------------------------------------------------------------- union-find */

static uint32_t uf_find(uint32_t *p, uint32_t x) {
  while (p[x] != x) { /* path halving */
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

/* returns 1 iff x and y were in different sets (they are merged) */
static int uf_union(uint32_t *p, uint32_t *sz, uint32_t x, uint32_t y) {
  x = uf_find(p, x);
  y = uf_find(p, y);
  if (x == y) return 0;
  if (sz[x] < sz[y]) {
    uint32_t t = x;
    x = y;
    y = t;
  }
  p[y] = x;
  sz[x] += sz[y];
  return 1;
}

/* Writes the ids whose bit is set, ascending, and returns how many. */
static uint64_t bits_to_ids(const uint8_t *flag, uint64_t m, uint32_t *out) {
  uint64_t k = 0;
  for (uint64_t e = 0; e < m; ++e)
    if (flag[e]) out[k++] = (uint32_t)e;
  return k;
}

/* ---------------------------------------------------------------- Kruskal */

/* Stable LSD radix sort of `ids` (given in ascending id order) by w[id], one
 * byte per pass; passes whose byte is equal for every element are skipped.
 * Because each pass is stable and the input is in id order, the result is in
 * (w, id) order. */
static int sort_ids_by_weight(uint32_t *ids, uint64_t k, const uint32_t *w) {
  uint32_t *tmp = (uint32_t *)malloc((k ? k : 1) * sizeof(uint32_t));
  if (!tmp) return 3;
  for (int shift = 0; shift < 32; shift += 8) {
    uint64_t cnt[257];
    memset(cnt, 0, sizeof(cnt));
    for (uint64_t i = 0; i < k; ++i) cnt[((w[ids[i]] >> shift) & 0xff) + 1]++;
    int trivial = 0;
    for (int b = 1; b <= 256; ++b)
      if (cnt[b] == k) trivial = 1;
    if (trivial) continue;
    for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
    for (uint64_t i = 0; i < k; ++i) tmp[cnt[(w[ids[i]] >> shift) & 0xff]++] = ids[i];
    memcpy(ids, tmp, k * sizeof(uint32_t));
  }
  free(tmp);
  return 0;
}

int oracle_kruskal(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                   uint32_t *out_ids, uint64_t *out_count, uint64_t *out_weight) {
  *out_count = 0;
  *out_weight = 0;
  if (n > 0xFFFFFFFFULL || m > 0xFFFFFFFFULL) return 2;
  if (check_range(n, m, src, dst)) return 1;
  uint32_t *order = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
  uint32_t *p = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint32_t *sz = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint8_t *in_f = (uint8_t *)calloc(m ? m : 1, 1);
  if (!order || !p || !sz || !in_f) {
    free(order);
    free(p);
    free(sz);
    free(in_f);
    return 3;
  }
  uint64_t k = 0;
  for (uint64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) order[k++] = (uint32_t)e; /* self-loops never join two trees */
  int rc = sort_ids_by_weight(order, k, w);
  if (rc == 0) {
    for (uint64_t v = 0; v < n; ++v) {
      p[v] = (uint32_t)v;
      sz[v] = 1;
    }
    uint64_t total = 0;
    for (uint64_t i = 0; i < k; ++i) {
      uint32_t e = order[i];
      if (uf_union(p, sz, src[e], dst[e])) {
        in_f[e] = 1;
        total += w[e];
      }
    }
    *out_count = bits_to_ids(in_f, m, out_ids);
    *out_weight = total;
  }
  free(order);
  free(p);
  free(sz);
  free(in_f);
  return rc;
}

/* ------------------------------------------------------------------- Prim */

typedef struct {
  uint64_t key;
  uint32_t vertex;
} heap_item;

static void heap_push(heap_item *h, uint64_t *len, heap_item it) {
  uint64_t i = (*len)++;
  while (i > 0) {
    uint64_t par = (i - 1) / 2;
    if (h[par].key <= it.key) break;
    h[i] = h[par];
    i = par;
  }
  h[i] = it;
}

static heap_item heap_pop(heap_item *h, uint64_t *len) {
  heap_item top = h[0], last = h[--(*len)];
  uint64_t i = 0;
  for (;;) {
    uint64_t c = 2 * i + 1;
    if (c >= *len) break;
    if (c + 1 < *len && h[c + 1].key < h[c].key) ++c;
    if (last.key <= h[c].key) break;
    h[i] = h[c];
    i = c;
  }
  if (*len > 0) h[i] = last;
  return top;
}

int oracle_prim(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint32_t *out_ids,
                uint64_t *out_count, uint64_t *out_weight) {
  *out_count = 0;
  *out_weight = 0;
  if (n > 0xFFFFFFFFULL || m > 0x7FFFFFFFULL) return 2;
  if (check_range(n, m, src, dst)) return 1;
  /* adjacency in CSR form: each non-self-loop edge appears at both endpoints */
  uint64_t *start = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
  uint32_t *adj = (uint32_t *)malloc((2 * m + 1) * sizeof(uint32_t));
  uint64_t *fill = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
  uint8_t *visited = (uint8_t *)calloc(n + 1, 1);
  uint8_t *in_f = (uint8_t *)calloc(m + 1, 1);
  heap_item *heap = (heap_item *)malloc((2 * m + 1) * sizeof(heap_item));
  int rc = 0;
  if (!start || !adj || !fill || !visited || !in_f || !heap) {
    rc = 3;
    goto done;
  }
  for (uint64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) {
      start[src[e] + 1]++;
      start[dst[e] + 1]++;
    }
  for (uint64_t v = 0; v < n; ++v) start[v + 1] += start[v];
  memcpy(fill, start, n * sizeof(uint64_t));
  for (uint64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) {
      adj[fill[src[e]]++] = (uint32_t)e;
      adj[fill[dst[e]]++] = (uint32_t)e;
    }
  uint64_t total = 0;
  for (uint64_t s = 0; s < n; ++s) {
    if (visited[s]) continue;
    uint64_t len = 0;
    visited[s] = 1;
    for (uint64_t i = start[s]; i < start[s + 1]; ++i) {
      uint32_t e = adj[i];
      uint32_t other = src[e] == s ? dst[e] : src[e];
      if (!visited[other]) heap_push(heap, &len, (heap_item){KEY(w[e], e), other});
    }
    while (len > 0) {
      heap_item it = heap_pop(heap, &len);
      if (visited[it.vertex]) continue; /* lazy deletion */
      uint32_t e = (uint32_t)(it.key & 0xFFFFFFFFULL);
      visited[it.vertex] = 1;
      in_f[e] = 1;
      total += w[e];
      uint32_t x = it.vertex;
      for (uint64_t i = start[x]; i < start[x + 1]; ++i) {
        uint32_t f = adj[i];
        uint32_t other = src[f] == x ? dst[f] : src[f];
        if (!visited[other]) heap_push(heap, &len, (heap_item){KEY(w[f], f), other});
      }
    }
  }
  *out_count = bits_to_ids(in_f, m, out_ids);
  *out_weight = total;
done:
  free(start);
  free(adj);
  free(fill);
  free(visited);
  free(in_f);
  free(heap);
  return rc;
}

/* ------------------------------------------------------------ brute force */

/* Tiny graphs only (n <= 16, m <= 22).  c = number of connected components.
 * Enumerates every edge subset of size n - c that contains no cycle (these are
 * exactly the spanning forests).  The forest minimising sum 2^rank(e), where
 * rank is the position in (w,id) order, is the unique order-minimal MSF, since
 * comparing such sums compares the sets' largest differing element.  Also
 * reports min sum w over all spanning forests, computed independently. */
int oracle_brute(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                 uint32_t *out_ids, uint64_t *out_count, uint64_t *out_weight, uint64_t *out_min_weight_any) {
  *out_count = 0;
  *out_weight = 0;
  *out_min_weight_any = 0;
  if (n > 16 || m > 22) return 2;
  if (check_range(n, m, src, dst)) return 1;
  uint32_t p[16], sz[16];
  for (uint32_t v = 0; v < n; ++v) {
    p[v] = v;
    sz[v] = 1;
  }
  uint64_t comps = n;
  for (uint64_t e = 0; e < m; ++e) comps -= (uint64_t)uf_union(p, sz, src[e], dst[e]);
  uint64_t need = n - comps;
  uint32_t rank[22];
  for (uint64_t e = 0; e < m; ++e) { /* rank = number of edges before e in (w,id) order */
    rank[e] = 0;
    for (uint64_t f = 0; f < m; ++f)
      if (KEY(w[f], f) < KEY(w[e], e)) rank[e]++;
  }
  uint64_t best_score = UINT64_MAX, best_set = 0, min_w = UINT64_MAX;
  for (uint64_t s = 0; s < (1ULL << m); ++s) {
    if ((uint64_t)__builtin_popcountll(s) != need) continue;
    for (uint32_t v = 0; v < n; ++v) {
      p[v] = v;
      sz[v] = 1;
    }
    int ok = 1;
    uint64_t score = 0, tw = 0;
    for (uint64_t e = 0; e < m && ok; ++e)
      if (s >> e & 1) {
        if (!uf_union(p, sz, src[e], dst[e])) ok = 0; /* cycle or self-loop */
        score += 1ULL << rank[e];
        tw += w[e];
      }
    if (!ok) continue;
    if (score < best_score) {
      best_score = score;
      best_set = s;
    }
    if (tw < min_w) min_w = tw;
  }
  uint64_t k = 0, total = 0;
  for (uint64_t e = 0; e < m; ++e)
    if (best_set >> e & 1) {
      out_ids[k++] = (uint32_t)e;
      total += w[e];
    }
  *out_count = k;
  *out_weight = total;
  *out_min_weight_any = need == 0 ? 0 : min_w;
  return 0;
}

/* ---------------------------------------------------------------- checks */

/* Checks that F (k ascending edge ids) is the MSF of G under the (w,id) order.
 * Returns a bit mask, 0 when every check passes:
 *   1  an id is out of range, repeated, unsorted, or a self-loop
 *   2  F contains a cycle
 *   4  |F| != n - c (F does not span every component)
 *   8  cut property fails: some e in F is not the (w,id)-minimum edge crossing
 *      the cut that removing e from its tree induces (Section 2.3, min-cut
 *      property)
 *  16  cycle property fails: some non-self-loop edge f not in F has endpoints
 *      unconnected in F or is not the (w,id)-maximum of the cycle it closes
 * Costs O(k (n + m) + m n); meant for graphs up to a few thousand vertices. */
int oracle_check_msf(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                     const uint32_t *ids, uint64_t k) {
  int bad = 0;
  if (check_range(n, m, src, dst)) return 1;
  uint8_t *in_f = (uint8_t *)calloc(m + 1, 1);
  uint32_t *p = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
  uint32_t *sz = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
  uint64_t *fstart = (uint64_t *)calloc(n + 2, sizeof(uint64_t));
  uint32_t *fadj = (uint32_t *)malloc((2 * k + 1) * sizeof(uint32_t));
  uint64_t *fill = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
  uint8_t *side = (uint8_t *)malloc(n + 1);
  uint32_t *stack = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
  uint32_t *par = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
  uint32_t *par_edge = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
  uint32_t *depth = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
  if (!in_f || !p || !sz || !fstart || !fadj || !fill || !side || !stack || !par || !par_edge || !depth) {
    bad = 64;
    goto done;
  }
  for (uint64_t i = 0; i < k; ++i) {
    if (ids[i] >= m || (i > 0 && ids[i] <= ids[i - 1]) || src[ids[i]] == dst[ids[i]]) {
      bad |= 1;
      goto done;
    }
    in_f[ids[i]] = 1;
  }
  /* acyclic and spanning */
  for (uint64_t v = 0; v < n; ++v) {
    p[v] = (uint32_t)v;
    sz[v] = 1;
  }
  for (uint64_t i = 0; i < k; ++i)
    if (!uf_union(p, sz, src[ids[i]], dst[ids[i]])) bad |= 2;
  if (bad) goto done;
  uint64_t comps = n;
  for (uint64_t v = 0; v < n; ++v) {
    p[v] = (uint32_t)v;
    sz[v] = 1;
  }
  for (uint64_t e = 0; e < m; ++e) comps -= (uint64_t)uf_union(p, sz, src[e], dst[e]);
  if (k != n - comps) {
    bad |= 4;
    goto done;
  }
  /* forest adjacency */
  for (uint64_t i = 0; i < k; ++i) {
    fstart[src[ids[i]] + 1]++;
    fstart[dst[ids[i]] + 1]++;
  }
  for (uint64_t v = 0; v < n; ++v) fstart[v + 1] += fstart[v];
  memcpy(fill, fstart, n * sizeof(uint64_t));
  for (uint64_t i = 0; i < k; ++i) {
    fadj[fill[src[ids[i]]]++] = ids[i];
    fadj[fill[dst[ids[i]]]++] = ids[i];
  }
  /* cut property */
  for (uint64_t i = 0; i < k && !(bad & 8); ++i) {
    uint32_t e = ids[i];
    memset(side, 0, n);
    uint64_t top = 0;
    stack[top++] = src[e];
    side[src[e]] = 1;
    while (top > 0) { /* vertices reachable from src[e] in F without e */
      uint32_t x = stack[--top];
      for (uint64_t j = fstart[x]; j < fstart[x + 1]; ++j) {
        uint32_t f = fadj[j];
        if (f == e) continue;
        uint32_t y = src[f] == x ? dst[f] : src[f];
        if (!side[y]) {
          side[y] = 1;
          stack[top++] = y;
        }
      }
    }
    for (uint64_t f = 0; f < m; ++f)
      if (f != e && side[src[f]] != side[dst[f]] && KEY(w[f], f) < KEY(w[e], e)) {
        bad |= 8;
        break;
      }
  }
  /* cycle property: root every tree, then compare against the path maximum */
  for (uint64_t v = 0; v < n; ++v) par[v] = UINT32_MAX;
  for (uint64_t r = 0; r < n; ++r) {
    if (par[r] != UINT32_MAX) continue;
    par[r] = (uint32_t)r;
    par_edge[r] = UINT32_MAX;
    depth[r] = 0;
    uint64_t top = 0;
    stack[top++] = (uint32_t)r;
    while (top > 0) {
      uint32_t x = stack[--top];
      for (uint64_t j = fstart[x]; j < fstart[x + 1]; ++j) {
        uint32_t f = fadj[j];
        uint32_t y = src[f] == x ? dst[f] : src[f];
        if (par[y] == UINT32_MAX) {
          par[y] = x;
          par_edge[y] = f;
          depth[y] = depth[x] + 1;
          stack[top++] = y;
        }
      }
    }
  }
  for (uint64_t f = 0; f < m && !(bad & 16); ++f) {
    if (in_f[f] || src[f] == dst[f]) continue;
    uint32_t a = src[f], b = dst[f];
    uint64_t pathmax = 0;
    while (a != b) {
      if (depth[a] < depth[b]) {
        uint32_t t = a;
        a = b;
        b = t;
      }
      if (par[a] == a) { /* different trees: f would connect two components of F */
        bad |= 16;
        break;
      }
      uint32_t pe = par_edge[a];
      if (KEY(w[pe], pe) > pathmax) pathmax = KEY(w[pe], pe);
      a = par[a];
    }
    if (!(bad & 16) && pathmax > KEY(w[f], f)) bad |= 16;
  }
done:
  free(in_f);
  free(p);
  free(sz);
  free(fstart);
  free(fadj);
  free(fill);
  free(side);
  free(stack);
  free(par);
  free(par_edge);
  free(depth);
  return bad;
}

/* --------------------------------------------------- Kruskal, parallel sort */

#define PAR_MAX_THREADS 256

/* One pass of the parallel stable radix sort: thread t owns the contiguous
 * chunk [lo, hi) of the current order and first counts its digits; after all
 * counts are known, every (digit, thread) pair gets its output start (digits
 * ascending, threads ascending within a digit: the order a sequential stable
 * pass would give), and each thread scatters its chunk in order. */
typedef struct {
  const uint32_t *w;
  const uint32_t *in;
  uint32_t *out;
  uint64_t lo, hi;
  int shift;
  uint64_t cnt[256];  /* digit counts of the chunk, then output starts */
} par_pass;

static void *par_count(void *arg) {
  par_pass *a = (par_pass *)arg;
  memset(a->cnt, 0, sizeof(a->cnt));
  for (uint64_t i = a->lo; i < a->hi; ++i) a->cnt[(a->w[a->in[i]] >> a->shift) & 0xff]++;
  return NULL;
}

static void *par_scatter(void *arg) {
  par_pass *a = (par_pass *)arg;
  for (uint64_t i = a->lo; i < a->hi; ++i) {
    const uint32_t id = a->in[i];
    a->out[a->cnt[(a->w[id] >> a->shift) & 0xff]++] = id;
  }
  return NULL;
}

/* Runs fn over the T pass records: records 1..T-1 on new threads, record 0
 * on the calling thread.  Returns 0, or 3 if a thread could not be started
 * (the records it would have run are then run here). */
static int par_run(void *(*fn)(void *), par_pass *rec, int T) {
  pthread_t th[PAR_MAX_THREADS];
  int started[PAR_MAX_THREADS];
  for (int t = 1; t < T; ++t) started[t] = pthread_create(&th[t], NULL, fn, &rec[t]) == 0;
  fn(&rec[0]);
  for (int t = 1; t < T; ++t) {
    if (started[t])
      pthread_join(th[t], NULL);
    else
      fn(&rec[t]);
  }
  return 0;
}

int oracle_kruskal_par(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                       int nthreads, uint32_t *out_ids, uint64_t *out_count, uint64_t *out_weight) {
  *out_count = 0;
  *out_weight = 0;
  if (n > 0xFFFFFFFFULL || m > 0xFFFFFFFFULL) return 2;
  if (check_range(n, m, src, dst)) return 1;
  int T = nthreads < 1 ? 1 : (nthreads > PAR_MAX_THREADS ? PAR_MAX_THREADS : nthreads);
  uint32_t *order = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
  uint32_t *tmp = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
  uint32_t *p = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint32_t *sz = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint8_t *in_f = (uint8_t *)calloc(m ? m : 1, 1);
  par_pass *rec = (par_pass *)malloc((size_t)T * sizeof(par_pass));
  if (!order || !tmp || !p || !sz || !in_f || !rec) {
    free(order);
    free(tmp);
    free(p);
    free(sz);
    free(in_f);
    free(rec);
    return 3;
  }
  uint64_t k = 0;
  for (uint64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) order[k++] = (uint32_t)e; /* self-loops never join two trees */
  if ((uint64_t)T > k) T = k > 0 ? (int)k : 1;
  for (int shift = 0; shift < 32; shift += 8) {
    for (int t = 0; t < T; ++t) {
      rec[t].w = w;
      rec[t].in = order;
      rec[t].out = tmp;
      rec[t].lo = k * (uint64_t)t / (uint64_t)T;
      rec[t].hi = k * (uint64_t)(t + 1) / (uint64_t)T;
      rec[t].shift = shift;
    }
    par_run(par_count, rec, T);
    uint64_t start = 0;
    int trivial = 0;
    for (int d = 0; d < 256; ++d) {
      uint64_t digit_total = 0;
      for (int t = 0; t < T; ++t) digit_total += rec[t].cnt[d];
      if (digit_total == k) trivial = 1;
    }
    if (trivial) continue; /* every element has the same digit: the pass keeps the order */
    for (int d = 0; d < 256; ++d)
      for (int t = 0; t < T; ++t) {
        const uint64_t c = rec[t].cnt[d];
        rec[t].cnt[d] = start;
        start += c;
      }
    par_run(par_scatter, rec, T);
    uint32_t *sw = order;
    order = tmp;
    tmp = sw;
  }
  for (uint64_t v = 0; v < n; ++v) {
    p[v] = (uint32_t)v;
    sz[v] = 1;
  }
  uint64_t total = 0;
  for (uint64_t i = 0; i < k; ++i) {
    const uint32_t e = order[i];
    if (uf_union(p, sz, src[e], dst[e])) {
      in_f[e] = 1;
      total += w[e];
    }
  }
  *out_count = bits_to_ids(in_f, m, out_ids);
  *out_weight = total;
  free(order);
  free(tmp);
  free(p);
  free(sz);
  free(in_f);
  free(rec);
  return 0;
}
