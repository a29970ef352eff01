/*
 * mst.h -- C ABI of libmstgpu, a single-GPU (GB300, sm_103a) minimum spanning
 * forest solver built on Borůvka rounds and Filter-Borůvka.
 *
 * Problem (Sanders & Schimek, "Engineering Massively Parallel MST Algorithms",
 * IPDPS 2023, Section 2.2): the input is an undirected weighted graph
 * G = (V, E) with n vertices and m edges; the output is a minimum spanning tree
 * of every connected component (a minimum spanning forest, MSF).  Here:
 *   - vertices are 0-based (the paper numbers them 1..|V|);
 *   - edge e is (src[e], dst[e], w[e]) with uint32 weight; its id is e;
 *   - the graph may hold self-loops (ignored) and parallel edges;
 *   - ties are broken by the strict total order (w, id) (Section 2.3: consistent
 *     tie breaking makes the MST unique), so the MSF is unique and the solver
 *     returns exactly its edge ids, ascending, plus the uint64 weight sum.
 *
 * Memory: every pointer named d_* is DEVICE memory on the handle's GPU, owned
 * by the caller; h_* pointers are host memory.  Device arrays must be 4-byte
 * aligned; 16-byte alignment enables vector loads.  The library allocates its
 * own scratch memory (stream-ordered) and frees it when the handle is destroyed.
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 * of a call's device work is issued on that stream, after the work the caller
 * queued on it before the call.  A call returns once its results are written:
 * the Borůvka round loop and the Filter-Borůvka recursion are steered by
 * counts (list lengths, active components) that the host reads back on that
 * stream, so a solve is stream-ordered but not asynchronous to the host.  A
 * handle must not be used by two host threads at once; different handles may
 * solve at the same time from different threads (each on its own stream): a
 * solve grows its buffers in stream order and never waits for the whole
 * device.  mst_create and mst_destroy do wait for the device, so create and
 * destroy handles while no other thread is capturing a CUDA graph.
 *
 * Errors: every call returns an mst_status.  Errors detected on the device
 * (vertex ids out of range, a bounded loop that ran out of iterations) are
 * read back before the call returns.  No call aborts the process.
 */
#ifndef MSTGPU_MST_H
#define MSTGPU_MST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mst_ctx *mst_handle;

typedef enum {
  MST_OK = 0,
  MST_ERR_INVALID_ARG = 1,  /* null pointer, bad config value */
  MST_ERR_VERTEX_RANGE = 2, /* some src[e] or dst[e] >= n */
  MST_ERR_TOO_LARGE = 3,    /* m >= 2^32 (edge ids are uint32) */
  MST_ERR_OOM = 4,          /* scratch allocation failed */
  MST_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  MST_ERR_INTERNAL = 6,     /* a bounded device loop ran out of iterations */
  MST_ERR_NOT_SUPPORTED = 7 /* option not available in this library */
} mst_status;

enum { MST_VARIANT_BORUVKA = 0, MST_VARIANT_FILTER = 1, MST_VARIANT_AUTO = 2 };
enum { MST_DEDUPE_AUTO = 0, MST_DEDUPE_SORT = 1, MST_DEDUPE_HASH = 2, MST_DEDUPE_NONE = 3 };

typedef struct {
  int device;                  /* CUDA device ordinal */
  int variant;                 /* MST_VARIANT_*: Borůvka (Alg. 1 rounds) or Filter-Borůvka (Alg. 2) */
  int dedupe;                  /* MST_DEDUPE_*: parallel-edge removal between rounds (Section 2.3, optional) */
  int tile_contract;           /* 0 off (default), 1 on, -1 auto (on when >= 10% of sampled edges are
                                  local): local contraction on vertex-range tiles before the rounds
                                  (Section 4.1).  Off by default: on one GPU its passes cost more than
                                  the global rounds they save, even on geometric graphs */
  uint32_t tile_vertices;      /* vertices per tile for local contraction, 32..4096 */
  uint32_t pivot_sample;       /* edges sampled per pivot selection (Alg. 2 PivotSelection) */
  uint64_t seed;               /* seed of the pivot sampling stream */
  uint64_t filter_min_edges;   /* isSparse: lists shorter than this are not partitioned */
  float filter_max_avg_degree; /* isSparse: stop partitioning at average degree 2m/n <= this (the paper's
                                  Section 6.3 uses 4; the default 1.25 is measured on GB300, where the range
                                  0.75-2.5 is flat with the default pivot quantile) */
  int base_case;               /* 1 (default): once a Borůvka call's live components (<= 4096) and
                                  edges (<= 6144) fit one block's shared memory, finish its rounds in
                                  one launch (the role of the paper's base case, Section 4.4); 0: run
                                  every round globally */
  int graph_rounds;            /* 1 (default): from the second round of a Borůvka call on, run the
                                  rounds as one CUDA graph launch whose conditional loop the device
                                  ends (no host round trip per round); 0: one host readback per round */
  int graph_jump_launches;     /* pointer-jumping launches per round inside the graph, 1..8, of up to
                                  256 parent steps each (default 2: chains up to 256^2); a round that
                                  needs more hands the state back to the host, which finishes the jump */
  int filter_carry;            /* Filter-Borůvka: 1 hands a level's filtered heavy edges, when at most
                                  n/8, back to the level above instead of solving them there (Section
                                  6.3); 0 (default, measured faster on GB300): every level solves its own */
  int filter_split;            /* Filter-Borůvka: 1 filters in two passes (heavy edges outside the giant
                                  component first, then the label test on that short list); 0 (default):
                                  one pass */
  int min_edges_sort;          /* 1: the first minEdges of a Borůvka call sorts both ends of every edge by
                                  vertex and takes segmented minima (one atomic per vertex run and warp, the
                                  sorted-edge form of Sections 2.2/4.5); 0 (default): one atomic pass */
  uint32_t jump_steps;         /* parent steps per pointer-jumping launch on the host-driven path,
                                  1..4096 (default 64); a launch that leaves a walk short is repeated
                                  (at most 64 more times, then MST_ERR_INTERNAL).  1 makes every launch
                                  one pointer-doubling step (Section 4.2) */
  int tile_filter;             /* 1: inside local contraction and the base case, the rounds use the light
                                  half of a tile's edges first and drop heavy edges that fall inside a
                                  component (recursive filtering in local preprocessing, Section 6.2);
                                  0 (default, measured faster on GB300): every edge from the first round */
  uint32_t spin_limit;         /* polls of a predecessor's status word in the ordered output scan before the
                                  wait gives up (>= 1; default 2^21, about a second); a wait that runs out
                                  makes the call return MST_ERR_INTERNAL.  Small values exist to exercise
                                  that error path */
  uint32_t block_threads;      /* threads per block of the relabel / partition compactions and the hooking
                                  kernel: 128, 256 or 512 (0 = 256) */
  uint32_t items_per_thread;   /* edges (or vertices) per thread of those kernels: 4, 8 or 16 (0 = 8); a
                                  block handles block_threads x items_per_thread per tile.  Both are
                                  autotuner choices; every shape computes the same forest */
  int filter_plan;             /* Filter-Borůvka (Alg. 2) with the default filter options (no carry, one
                                  filter pass, CUDA-graph rounds, no dedupe, no local contraction):
                                  1 (default): after the top-level partition, the host plans the
                                  remaining recursion levels and list capacities from its light count
                                  and queues every level without reading counts back (lengths stay in
                                  device memory; Borůvka rounds run as device-ended graph loops); the
                                  call reads back twice.  If a list outgrows its planned capacity or a
                                  round needs the host, the call starts over on the host-driven path
                                  (same result).  0: the host reads every level's counts */
  uint32_t relabel_block_threads;    /* threads per block of the relabel compaction, which runs in every
                                        Borůvka round, mostly on short lists: 128, 256 or 512; both
                                        relabel fields 0: 128 x 4, measured fastest on GB300 (more,
                                        smaller tiles spread a short list over more SMs) */
  uint32_t relabel_items_per_thread; /* edges per thread of the relabel compaction: 4, 8 or 16 */
  float pivot_quantile;        /* Filter-Borůvka: the pivot is the sample key of rank floor(q * pivot_sample),
                                  so about a share q of each list is light (Alg. 2 PivotSelection takes the
                                  median, q = 0.5).  1/64 <= q <= 1/2.  A smaller q writes shorter light lists
                                  and needs fewer recursion levels, while the filter meets more heavy edges
                                  (over all levels about the same number); every q computes the same forest.
                                  Default 0.125, measured on GB300: RMAT n=2^24 m=2^28 took 7.16 / 5.54 /
                                  5.25 / 5.35 ms at q = 1/2, 1/4, 1/8, 1/16 (flat from 3/32 to 5/32; all
                                  with the block-kernel partition, which runs for q > 1/8), 4.90 ms at 1/8
                                  with the warp-streamed partition */
} mst_config;

/* Fills *cfg with the defaults (Borůvka variant, automatic dedupe, pivot sample
 * 2^16 split at its 1/8 quantile, isSparse average degree 1.25, lists below
 * 2^20 edges not partitioned). */
void mst_config_default(mst_config *cfg);

/* Creates a handle on cfg->device (cfg == NULL: defaults on device 0). */
mst_status mst_create(mst_handle *out, const mst_config *cfg);

/* Frees the handle and all of its device memory.  NULL is ignored. */
void mst_destroy(mst_handle h);

/* Replaces the handle's configuration. */
mst_status mst_set_config(mst_handle h, const mst_config *cfg);

/* Human-readable name of a status code (static storage). */
const char *mst_status_string(mst_status s);

/* Waits for `stream`, then returns the status of the last call made with
 * this handle, or, if that call succeeded, the error flags the device has
 * latched since it began (vertex range, an exhausted bounded loop), as a
 * status.  MST_ERR_CUDA if the stream reports a CUDA error. */
mst_status mst_get_error(mst_handle h, void *stream);

/* The CUDA runtime error code (cudaError_t) behind the last MST_ERR_CUDA
 * returned for this handle, 0 if none; *line (if line != NULL) receives the
 * library source line of the failing call, 0 if unknown.  For diagnostics. */
int mst_last_cuda_error(mst_handle h, int *line);

/* Upper bound on the scratch bytes a solve of (n, m) allocates with the given
 * configuration (cfg == NULL: defaults), for admission by memory footprint. */
uint64_t mst_workspace_bytes(uint32_t n, uint64_t m, const mst_config *cfg);

/* Minimum spanning forest of the graph (n, m, d_src, d_dst, d_w)
 * (Section 2.2 problem; Borůvka rounds of Section 2.3 / Alg. 1, or Alg. 2).
 *   d_msf_ids       [out] capacity >= min(m, max(n-1, 0)); receives the MSF
 *                   edge ids in ascending order
 *   d_msf_count     [out] one uint32: number of ids written
 *   d_total_weight  [out] one uint64: sum of w over the MSF
 * n = 0 or m = 0 gives an empty forest of weight 0.  Inputs are not modified. */
mst_status mst_solve(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                     const uint32_t *d_w, uint32_t *d_msf_ids, uint32_t *d_msf_count, uint64_t *d_total_weight,
                     void *stream);

/* As mst_solve, with every array in HOST memory: the call copies the inputs to
 * the device, solves, and copies the forest back before returning.
 * h_msf_ids needs capacity min(m, max(n-1, 0)). */
mst_status mst_solve_host(mst_handle h, uint32_t n, uint64_t m, const uint32_t *h_src, const uint32_t *h_dst,
                          const uint32_t *h_w, uint32_t *h_msf_ids, uint32_t *h_msf_count, uint64_t *h_total_weight,
                          void *stream);

/* One graph in HOST memory for mst_solve_host_many: inputs as mst_solve (src,
 * dst, w: m entries each; page-locked memory copies fastest), results as
 * mst_solve_host (msf_ids: capacity min(m, max(n-1, 0)), ascending ids). */
typedef struct {
  uint32_t n;
  uint64_t m;
  const uint32_t *src, *dst, *w;
  uint32_t *msf_ids;      /* [out] */
  uint32_t msf_count;     /* [out] */
  uint64_t total_weight;  /* [out] */
  mst_status status;      /* [out] this graph's status */
} mst_host_graph;

/* Solves graphs[0..count-1] in order, each as mst_solve_host, with the copy of
 * graph i+1's inputs to the device overlapping the solve of graph i (two
 * device input buffers, a copy stream of the handle; the solves run on
 * `stream`), so a sequence of host-resident graphs costs about max(copy, solve)
 * per graph rather than their sum.  Each graph gets its own status; a graph
 * that fails with MST_ERR_CUDA or MST_ERR_OOM ends the sequence, and the
 * graphs after it keep status MST_ERR_INTERNAL (not attempted).  Returns
 * MST_OK if every graph was solved, else the first failing graph's status. */
mst_status mst_solve_host_many(mst_handle h, uint32_t count, mst_host_graph *graphs, void *stream);

/* Minimum spanning forests of G independent graphs in one solve (each graph
 * the Section 2.2 problem).  Graph g has d_n[g] vertices (graph-local ids
 * 0..d_n[g]-1) and the edges d_edge_off[g] .. d_edge_off[g+1]-1 of
 * d_src/d_dst/d_w.  The graphs are solved together as one disjoint union, so
 * their rounds share launches.
 *   d_n         [G] uint32 vertex counts, device memory
 *   d_edge_off  [G+1] uint64 edge offsets, device memory; d_edge_off[0] == 0,
 *               non-decreasing (else MST_ERR_INVALID_ARG); d_edge_off[G] = m
 *   d_msf_ids   [out] capacity >= sum_g min(m_g, n_g - 1) (min(m, sum_g n_g)
 *               always suffices); segment g starts at d_msf_off[g] and holds
 *               graph-local edge ids (index - d_edge_off[g]), ascending
 *   d_msf_off   [out] [G+1] uint64 segment offsets
 *   d_total_weight [out] [G] uint64 MSF weight of each graph
 * The totals (all vertices, all edges) are read back from the device tables
 * before the solve is sized.  MST_ERR_TOO_LARGE if either reaches 2^32.
 * Errors as mst_solve; a vertex id out of range in any graph fails the call. */
mst_status mst_solve_batched(mst_handle h, uint32_t num_graphs, const uint32_t *d_n, const uint64_t *d_edge_off,
                             const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w, uint32_t *d_msf_ids,
                             uint64_t *d_msf_off, uint64_t *d_total_weight, void *stream);

/* Per-kernel-class timing: when enabled, every kernel launch of a solve is
 * bracketed by CUDA events on the solve's stream, and the elapsed time,
 * launch count and algorithmic bytes (the bytes the method must move: edge
 * records read and written, vertex arrays; label gathers, atomics and hash
 * probes are not counted) are accumulated per class until reset. */
enum {
  MST_K_MIN_EDGES = 0,  /* minEdges from a stored list (first round of a Borůvka call) */
  MST_K_RELABEL_MIN,    /* relabel + self-loop removal + compaction, fused with the next minEdges */
  MST_K_HOOK,           /* hooking + active-vertex compaction */
  MST_K_JUMP,           /* pointer doubling */
  MST_K_DEDUPE,         /* hash parallel-edge removal (insert and keep passes) */
  MST_K_PIVOT,          /* pivot sampling and selection */
  MST_K_PARTITION,      /* light/heavy partition */
  MST_K_FILTER,         /* filtering of heavy edges */
  MST_K_FINALIZE,       /* bitmap -> ascending ids + weight */
  MST_K_TILE,           /* tile-local contraction (count, bucket, contract) */
  MST_K_BASE,           /* single-block base case (the last rounds of a Borůvka call) */
  MST_K_GRAPH,          /* Borůvka rounds run as one CUDA graph launch (time only; bytes not counted) */
  MST_K_COUNT
};
typedef struct {
  uint64_t launches;
  double ms;        /* summed event time of the class's launches */
  double bytes;     /* summed algorithmic bytes of the passes as built */
  double min_bytes; /* summed bytes the method itself must move: equal to `bytes` except for the
                       filter, whose pass also re-reads the light edges of its list (the paper's
                       filter reads only the heavy edges, Alg. 2): there the heavy edges read
                       plus the survivors written */
} mst_kernel_stats;

/* enable != 0: start collecting (and clear the totals); 0: stop. */
mst_status mst_profile_enable(mst_handle h, int enable);

/* Classes (bit MST_K_x) timed with CUDA events while profiling; the others
 * only count their launches and algorithmic bytes, which costs the host almost
 * nothing per launch.  Default: all classes. */
mst_status mst_profile_classes(mst_handle h, uint32_t mask);

/* Totals of class `kind` (MST_K_*) since the last enable. */
mst_status mst_profile_get(mst_handle h, int kind, mst_kernel_stats *out);

/* Host-side counters of a handle since its creation (always on). */
typedef struct {
  uint64_t solves;         /* solves that reached the device (a batched solve counts once) */
  uint64_t readbacks;      /* times the host waited for device counts (each ends the GPU's queue for a
                              few microseconds; the planned Filter-Borůvka needs two per solve) */
  uint64_t planned;        /* solves that took the planned Filter-Borůvka path (mst_config.filter_plan) */
  uint64_t plan_fallbacks; /* of those, solves whose plan did not hold and that started over on the
                              host-driven path */
} mst_host_counters;
mst_status mst_host_counters_get(mst_handle h, mst_host_counters *out);

/* ----------------------------------------------------------------------
 * Step entry points: one step of the method each, on caller buffers, so that
 * every step can be checked on its own.  Edge lists are SoA (u, v, w, id) of
 * length m; d_id may be NULL, meaning id = index.  "key" means the uint64
 * (w << 32) | id.  The list-producing steps write their survivors in an
 * unspecified order (tiles land in the order they finish); the set of
 * survivors is exact.
 * -------------------------------------------------------------------- */

/* minEdges (Alg. 1; Section 2.3): d_best[c] = minimum key over the
 * non-self-loop edges incident to vertex c, or 2^64-1 if none.  d_best: [n]. */
mst_status mst_step_min_edges(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                              const uint32_t *d_w, const uint32_t *d_id, uint64_t *d_best, void *stream);

/* Hook + pointer doubling (Section 2.3; Section 4.2 contractComponents) of one
 * round: every vertex with an incident edge hooks to the other end of its
 * minimum edge; a 2-cycle keeps the smaller vertex as root; pointers are then
 * doubled until every tree is a star.  d_id must be NULL (edge id = index).
 *   d_parent   [out] [n] root of every vertex (itself when it has no edge)
 *   d_chosen   [in/out] bitmap over edge ids (bit id%32 of word id/32); the
 *              bits of the chosen edges are set, each edge once */
mst_status mst_step_contract(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                             const uint32_t *d_w, const uint32_t *d_id, uint32_t *d_parent, uint32_t *d_chosen,
                             void *stream);

/* Relabel (Section 4.3): (u, v) -> (d_label[u], d_label[v]); self-loops are
 * dropped.  Output arrays need capacity m; d_out_count receives one uint64. */
mst_status mst_step_relabel(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                            const uint32_t *d_w, const uint32_t *d_id, const uint32_t *d_label, uint32_t *d_ou,
                            uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid, uint64_t *d_out_count, void *stream);

/* Parallel-edge removal (Section 2.3; Section 4.3 Redistribute; Section 6.2
 * hash table): of the edges joining one unordered pair keep the minimum key;
 * survivors keep their orientation.  Capacity m; one uint64 count. */
mst_status mst_step_dedupe(mst_handle h, uint64_t m, const uint32_t *d_u, const uint32_t *d_v, const uint32_t *d_w,
                           const uint32_t *d_id, uint32_t *d_ou, uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid,
                           uint64_t *d_out_count, void *stream);

/* PivotSelection (Alg. 2; Section 5): sample k = 0..sample-1 is the edge at
 * position floor(splitmix64(state, k) * m / 2^64), where splitmix64(s, k) is
 * output k of the splitmix64 sequence started at state s; the pivot is the
 * sample key of rank sample/2 (0-based, ascending).  d_pivot: one uint64.
 * MST_ERR_TOO_LARGE if m >= 2^32 (edge ids are uint32). */
mst_status mst_step_pivot(mst_handle h, uint64_t m, const uint32_t *d_w, const uint32_t *d_id, uint64_t state,
                          uint32_t sample, uint64_t *d_pivot, void *stream);

/* Light part of the partition (Alg. 2): edges with key <= pivot and u != v.
 * Capacity m; one uint64 count. */
mst_status mst_step_partition(mst_handle h, uint64_t m, const uint32_t *d_u, const uint32_t *d_v, const uint32_t *d_w,
                              const uint32_t *d_id, uint64_t pivot, uint32_t *d_ou, uint32_t *d_ov, uint32_t *d_ow,
                              uint32_t *d_oid, uint64_t *d_out_count, void *stream);

/* Filter (Alg. 2; Section 5): edges with key > pivot, relabelled by the
 * representative array d_P after pointer doubling it to its roots (d_P is
 * updated in place to the roots); edges inside one component are dropped.
 * Capacity m; one uint64 count.  Every d_P[x] must be < n and the pointers
 * must lead to roots (d_P[r] == r): an entry >= n is MST_ERR_VERTEX_RANGE
 * (checked before d_P is used; d_P is then unchanged), a cycle longer than one
 * is MST_ERR_INTERNAL after a bounded number of pointer-jumping launches. */
mst_status mst_step_filter(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                           const uint32_t *d_w, const uint32_t *d_id, uint64_t pivot, uint32_t *d_P, uint32_t *d_ou,
                           uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid, uint64_t *d_out_count, void *stream);

/* Local preprocessing (Section 4.1) with vertex-range tiles in place of PEs:
 * vertex x is in tile x / tile_vertices (32..4096); an edge with both ends in
 * one tile is local.  Borůvka rounds run on each tile's local edges, and a
 * component is contracted along its lightest local edge only if that edge is
 * lighter than every cut edge incident to the component; rounds repeat until
 * no component contracts.
 *   d_parent  [out] [n] tile root of every vertex
 *   d_chosen  [in/out] bitmap over edge ids; bits of contracted edges are set
 * Input as mst_solve (validated; MST_ERR_VERTEX_RANGE on a bad id). */
mst_status mst_step_tile_contract(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                                  const uint32_t *d_w, uint32_t tile_vertices, uint32_t *d_parent, uint32_t *d_chosen,
                                  void *stream);

/* Output step (Section 2.2 output; Section 6.2 edge ids): the set bits of the
 * bitmap d_chosen over ids 0..m-1 become ascending ids in d_msf_ids, their
 * count in d_msf_count (uint32) and their weight sum over d_w in
 * d_total_weight (uint64). */
mst_status mst_step_finalize(mst_handle h, uint64_t m, const uint32_t *d_chosen, const uint32_t *d_w,
                             uint32_t *d_msf_ids, uint32_t *d_msf_count, uint64_t *d_total_weight, void *stream);

/* ----------------------------------------------------------------------
 * Allocation-free pivot selection.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code running
 * where cudaMalloc must not be called (host callbacks, real-time threads that
 * may not block on the allocator), or callers that reserve all of their device
 * memory themselves and so cannot create a handle (mst_create allocates).
 *
 * Computes exactly what mst_step_pivot computes (same sampling rule, same
 * rank), but needs no handle and calls no allocator: its scratch (the sampled
 * keys) is a fixed device array of MST_PIVOT_NOALLOC_MAX_SAMPLE uint64 entries
 * (512 KiB) inside the library, which every GPU that loads the library holds
 * until the process exits.
 *   m, d_w, d_id, state, sample  as in mst_step_pivot (d_id may be NULL)
 *   d_pivot  [out] one uint64, device memory, written in stream order
 * Runs on the current CUDA device and returns without waiting for the GPU.
 * The first call on a device looks the array's device address up once (with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture.  cudaDeviceReset on that device after
 * the first call is not supported (the array may move and the kept address
 * would be stale).  An error that earlier work on the calling thread left
 * pending (cudaPeekAtLastError) makes the call return MST_ERR_CUDA without
 * launching; the pending error is left in place for its owner.
 * All calls share the one array and it keeps the last call's samples: calls
 * whose work overlaps on the GPU (different streams, or different host threads
 * without ordering) race on it and may return wrong pivots.
 * Errors: MST_ERR_TOO_LARGE if sample > MST_PIVOT_NOALLOC_MAX_SAMPLE or
 * m >= 2^32; MST_ERR_INVALID_ARG for a NULL output, NULL d_w with m > 0 or
 * sample == 0; MST_ERR_CUDA if the address lookup or the launch fails. */
#define MST_PIVOT_NOALLOC_MAX_SAMPLE 65536u
mst_status mst_pivot_noalloc(uint64_t m, const uint32_t *d_w, const uint32_t *d_id, uint64_t state, uint32_t sample,
                             uint64_t *d_pivot, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MSTGPU_MST_H */
