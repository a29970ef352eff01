// Internal interfaces between the host solver (solver.cu) and the kernels
// (kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mstgpu {

typedef unsigned long long u64;
constexpr u64 KEY_INF = ~0ULL;

// Device-side error bits, latched in DevState::err.
enum : uint32_t {
  ERR_VERTEX = 1u,    // an input vertex id >= n
  ERR_LOOKBACK = 2u,  // a scan predecessor never published (bounded wait ran out)
  ERR_HASH = 4u,      // hash table probe sequence exhausted
  ERR_JUMP = 8u,      // pointer doubling did not reach a root within its bound
  ERR_TMA = 16u,      // a bulk copy never completed (bounded mbarrier wait ran out); tiles were skipped
  ERR_TABLE = 32u,    // a batched size table is inconsistent (offsets not starting at 0 or decreasing)
  ERR_OVERFLOW = 64u, // a compaction's survivors exceeded its output capacity (nothing past it was written)
  ERR_HANDBACK = 128u,  // device-driven rounds met a case that needs the host (long jump chain, round bound)
};

// Small per-handle device state.
constexpr int LVL_MAX = 32;  // recursion levels of a planned Filter-Borůvka
struct DevState {
  uint32_t err;
  uint32_t jump_flag;   // set when a pointer-jump launch left a vertex short of its root
  uint32_t tile_ctr[2]; // reserved
  u64 count[6 + 2 * LVL_MAX];  // counts written by the last tile of a scan kernel; from CNT_LVL on,
                               //   the list lengths of a planned Filter-Borůvka (see CNT_LVL)
  u64 pivot;            // result of the pivot selection
  uint32_t giant_root;  // root of the largest sampled component (filter fast path)
  uint32_t max_w;       // largest input weight (key layout)
  uint32_t local_samples;  // sampled local edges (automatic tile contraction)
  uint32_t giant_count;    // of the GIANT_SAMPLES sampled edge ends, those in the giant component
};
// Edge ends the giant-component root is sampled from.  The filter tests the
// giant-component bitmap first only when at least GIANT_MIN_COUNT of them lie
// in that component: otherwise (a batch of many small graphs has no giant
// component) nearly every heavy edge needs its labels anyway, and the bitmap
// gathers only add a dependent round trip.
constexpr uint32_t GIANT_SAMPLES = 1024, GIANT_MIN_COUNT = 512;
// CNT_LVL + k: length of the light list of recursion level k (level 0: the
// input); CNT_LVL + LVL_MAX + k: the filtered heavy edges of level k.
enum { CNT_EDGES = 0, CNT_ACTIVE = 1, CNT_TMP = 2, CNT_AUX = 3, CNT_USER = 4, CNT_CUT = 5, CNT_LVL = 6 };

// Output bookkeeping of a compaction launch.  Unordered compactions claim
// their output ranges by atomic adds on *total (zero before the launch); the
// ordered scan of the output ids uses the look-back status words, and its last
// tile writes *total.
struct ScanState {
  u64 *status;       // one status word per tile: epoch(30) | flag(2) | value(32)
  uint32_t *tile_ctr;  // unused
  uint32_t epoch;    // 1 .. 2^30-1, different for every ordered launch
  u64 *total;
  uint32_t *err;
  uint32_t spin_limit;  // polls of a predecessor's status word before the wait gives up (ERR_LOOKBACK)
};

struct HashSlot {
  u64 pair;  // (min(u,v) << 32) | max(u,v); all ones = empty
  u64 key;   // minimum (w << 32) | id seen for this pair
};

// Layout of the uint64 relaxation key of a solve.  Edges are ordered by
// (w, id).  When the weight, the edge id and a vertex id fit into 64 bits
// together (vbits + idbits + bits(max w) <= 64), the key is
//   w << (idbits + vbits) | id << vbits | other,
// where `other` is the far end of the edge as seen from the relaxed vertex, so
// the hook reads the chosen neighbour straight from the key.  Otherwise the
// key is w << 32 | id and the hook finds the neighbour through the input
// arrays.  Either way the minimum key of a vertex is its (w, id)-lightest edge.
struct KeyLayout {
  int packed;
  int vbits, idbits;
};

// An edge list in structure-of-arrays form.  id == nullptr: id = index.
struct EdgeList {
  const uint32_t *u, *v, *w, *id;
};
struct EdgeOut {
  uint32_t *u, *v, *w, *id;
};

enum CompactMode : int {
  CM_RELABEL = 0,    // (label[u], label[v]); drop self-loops
  CM_PARTITION = 1,  // key <= pivot and u != v; unchanged
  CM_FILTER = 2,     // key > pivot; (label[u], label[v]); drop self-loops
  CM_DEDUPE = 3,     // keep iff the hash table holds this edge's key for its pair
  CM_HEAVY = 4,      // key > pivot and not both ends in the giant component; unchanged (first filter pass)
};

struct CompactArgs {
  EdgeList in;
  uint64_t m;              // input length, or with m_dev the input list's capacity
  const u64 *m_dev;        // input length in device memory (read as min(*m_dev, m)), or nullptr
  EdgeOut out;
  const uint32_t *label;   // relabel / filter
  const uint32_t *giant_bits;  // filter: bitmap of the vertices in the largest component, or nullptr
  const uint32_t *giant_count; // filter: if set, the bitmap is used only when *giant_count >= GIANT_MIN_COUNT
  u64 pivot;               // partition / filter (used when pivot_dev == nullptr)
  const u64 *pivot_dev;
  u64 *best;               // if set: relax best[] of both ends with each survivor's key
  KeyLayout kl;
  HashSlot *table;         // dedupe lookup, or insert target when hash_insert
  uint64_t tmask;
  int hash_insert;
  uint32_t n;              // vertex count, for validation
  int validate;            // check u, v < n (sets ERR_VERTEX, skips the edge)
  uint32_t *max_w;         // if set: atomicMax of every input weight (key layout)
  uint32_t *cur_u, *cur_v; // if set: cur_u[id], cur_v[id] = the survivor's written ends
  ScanState st;
  int shape;               // tile shape of the relabel / partition compaction (see shape_index)
  int warp_partition;      // partition in the default shape: 1 runs the warp-streamed pass (for light
                           //   shares up to 1/8, where its per-warp output claims stay few), 0 the block kernel
  uint64_t out_cap;        // if nonzero: output capacity; a tile that would write past it writes
                           //   nothing and sets ERR_OVERFLOW (with m_dev, m bounds the input count)
};

struct HookArgs {
  const uint32_t *cand;    // candidate vertices; nullptr = 0..ncand-1
  uint64_t ncand;
  const u64 *ncand_dev;    // candidate count in device memory, or nullptr
  u64 *best;               // keys (see KeyLayout) of the round's minimum edges
  KeyLayout kl;
  const uint32_t *src, *dst;  // ends of each edge by id (unpacked keys): the input arrays,
                              // or the ends recorded when the current list was written
  uint32_t *parent;
  uint32_t *chosen_bits;   // bitmap over edge ids
  uint32_t *active_out;    // active vertices (best != INF), unspecified order
  u64 *counter;            // number written to active_out; zero before the launch
  uint32_t *err;
  u64 *wsum;               // if set: the weights of the chosen edges are added into these
                           //   WSUM_SLOTS counters (one add per warp, spread over the slots)
  int shape;               // tile shape (see shape_index)
};

// Tile shapes of the compaction and hook kernels, as the `shape` field of
// their argument structs: 0 is the default, 256 threads per block x 8 items
// per thread (so a zero-initialised struct gets it); 1 + 3 * b + i is the b-th
// of {128, 256, 512} threads with the i-th of {4, 8, 16} items per thread.
constexpr int SHAPE_COUNT = 10;
inline int shape_index(uint32_t block_threads, uint32_t items_per_thread) {
  if (block_threads == 0 && items_per_thread == 0) return 0;
  const uint32_t bt = block_threads ? block_threads : 256, it = items_per_thread ? items_per_thread : 8;
  const int b = bt == 128 ? 0 : bt == 256 ? 1 : bt == 512 ? 2 : -1;
  const int i = it == 4 ? 0 : it == 8 ? 1 : it == 16 ? 2 : -1;
  return (b < 0 || i < 0) ? -1 : 1 + 3 * b + i;
}
// The relabel compaction's shape: both zero is 128 x 4 (shape 1).
inline int relabel_shape_index(uint32_t block_threads, uint32_t items_per_thread) {
  return (block_threads == 0 && items_per_thread == 0) ? 1 : shape_index(block_threads, items_per_thread);
}
inline uint32_t shape_tile(int shape) {
  static const uint32_t b[3] = {128, 256, 512}, i[3] = {4, 8, 16};
  return shape <= 0 ? 2048u : b[(shape - 1) / 3] * i[(shape - 1) % 3];
}

// Counters the kernels that choose MSF edges add the chosen weights into, so
// that the forest's total needs no gather of w at the end.
constexpr int WSUM_SLOTS = 256;

// ---- launchers (kernels.cu); all asynchronous on `s` ----
int max_scan_tiles(uint64_t count);
void launch_compact(CompactMode mode, const CompactArgs &a, uint64_t max_count, cudaStream_t s);
void launch_min_edges(EdgeList in, uint64_t m, uint32_t n, int validate, KeyLayout kl, u64 *best, uint32_t *err,
                      int sms, cudaStream_t s);
void launch_max_weight(const uint32_t *w, uint64_t m, uint32_t *out, int sms, cudaStream_t s);
void launch_hook(const HookArgs &a, uint64_t max_cand, cudaStream_t s);
// max_steps: parent steps per thread and launch (0: the default of 64).
// With act == count_dev == nullptr the launch covers every vertex
// 0..count_host-1 and, given gbits, sets bit v of that bitmap iff v's walk
// reached the root *groot in this launch (gbits is ignored for lists).
void launch_jump(const uint32_t *act, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                 uint32_t *parent, u64 *best, int reset_best, uint32_t *flag, int sms, cudaStream_t s,
                 uint32_t max_steps = 0, const uint32_t *groot = nullptr, uint32_t *gbits = nullptr);
// Sets ERR_VERTEX in *err if some x[i] (i < count) is >= bound.
void launch_range_check(const uint32_t *x, uint64_t count, uint32_t bound, uint32_t *err, int sms, cudaStream_t s);
void launch_hash_insert(EdgeList in, uint64_t m, HashSlot *table, uint64_t tmask, uint32_t *err, int sms,
                        cudaStream_t s);
// The pivot is the sample key of rank `rank` (0-based); a rank >= sample
// means sample / 2, the sample median of Alg. 2.
void launch_pivot(EdgeList in, uint64_t m, const u64 *m_dev, u64 state, uint32_t sample, u64 *sample_buf,
                  u64 *pivot_out, cudaStream_t s, uint32_t rank = ~0u);
// Pivot selection by a cooperative multi-block radix select (same result as
// launch_pivot); `scratch` holds pivot_scratch_bytes().  False if the
// cooperative launch was refused.
size_t pivot_scratch_bytes();
bool launch_pivot_coop(EdgeList in, uint64_t m, u64 state, uint32_t sample, u64 *keys, void *scratch,
                       u64 *pivot_out, cudaStream_t s, const u64 *m_dev = nullptr, uint32_t rank = ~0u);
// w == nullptr: ids and count only (total_weight untouched).
void launch_finalize(const uint32_t *bits, uint64_t m, const uint32_t *w, uint32_t *out_ids, uint32_t *out_count,
                     u64 *total_weight, ScanState st, cudaStream_t s);
// *total = the sum of the WSUM_SLOTS counters.
void launch_wsum_total(const u64 *wsum, u64 *total, cudaStream_t s);
// The giant component's root: the most frequent root among the labels of
// sampled edge ends (P is walked to the roots); launch_giant_bits also marks
// its vertices (bit v set iff P[v] is that root; P fully contracted).
void launch_giant_root(EdgeList in, uint64_t m, u64 state, const uint32_t *P, uint32_t n, uint32_t *root_tmp,
                       cudaStream_t s, const u64 *m_dev = nullptr, uint32_t *count_out = nullptr);
void launch_giant_bits(EdgeList in, uint64_t m, u64 state, const uint32_t *P, uint32_t n, uint32_t *root_tmp,
                       uint32_t *bits, int sms, cudaStream_t s);
// tile-local contraction (Section 4.1)
void launch_tile_count(EdgeList in, uint64_t m, uint32_t n, uint32_t B, u64 *cutmin, uint32_t *count,
                       u64 *local_total, uint32_t *max_w, uint32_t *err, int sms, cudaStream_t s);
void launch_tile_scan(const uint32_t *count, uint32_t ntiles, u64 *offsets, cudaStream_t s);
void launch_tile_scatter(EdgeList in, uint64_t m, uint32_t n, uint32_t B, const u64 *offsets, uint32_t *fill,
                         uint32_t *b_ends, uint32_t *b_w, uint32_t *b_id, EdgeOut cut, u64 *cut_fill, int sms,
                         cudaStream_t s);
bool launch_tile_contract(uint32_t n, uint32_t B, uint64_t nlocal, const u64 *cutmin, const u64 *offsets,
                          const uint32_t *b_ends, const uint32_t *b_w, const uint32_t *b_id, uint32_t *parent,
                          uint32_t *bits, EdgeOut rest, u64 *rest_fill, uint32_t *err, cudaStream_t s,
                          int filter_heavy, u64 *wsum);
void launch_tile_sample(EdgeList in, uint64_t m, uint32_t n, uint32_t B, u64 state, uint32_t samples,
                        uint32_t *local_count, cudaStream_t s);
// Stable LSD radix sort of (u64 key, u32 value) pairs over the low `bits` bits;
// true when the result is in (keys_tmp, vals_tmp).  hist holds radix_hist_bytes().
size_t radix_hist_bytes(uint64_t m, int sms);
bool launch_radix_sort(u64 *keys, uint32_t *vals, u64 *keys_tmp, uint32_t *vals_tmp, uint64_t m, int bits,
                       uint32_t *hist, int sms, cudaStream_t s);
// Sort-based parallel-edge removal of list T (ends already component labels,
// no self-loops, ids present): keeps each unordered pair's (w, id)-lightest
// edge and emits it through `emit` (out, counter, best / ends as a compaction).
// vbits: bits of a vertex label; wbits, ibits: of a weight and an id.
size_t sort_dedupe_scratch_bytes(uint64_t m, int sms);
void launch_sort_dedupe(EdgeList T, uint64_t m, int vbits, int wbits, int ibits, const CompactArgs &emit,
                        void *scratch, int sms, cudaStream_t s);

// minEdges by sorting both ends of every edge by vertex and taking segmented
// minima (one atomic per vertex run and warp); false if 2m does not fit 32 bits.
size_t min_edges_sort_scratch_bytes(uint64_t m, int sms);
bool launch_min_edges_sort(EdgeList E, uint64_t m, uint32_t n, int validate, KeyLayout kl, u64 *best, uint32_t *err,
                           void *scratch, int sms, cudaStream_t s);

// Borůvka rounds as a CUDA graph (device-driven loop): state in device memory.
enum : uint32_t { ROUNDS_RUNNING = 0xff, ROUNDS_DONE = 0, ROUNDS_BASE = 1, ROUNDS_JUMP = 2, ROUNDS_BOUND = 3 };
struct GraphRounds {
  u64 ce[2];      // edges in the list of slot 0 / 1
  u64 ca[2];      // active vertices of slot 0 / 1
  u64 saved_ce, saved_ca;  // counts of the slot handed back to the host
  uint32_t jflag; // the round's last jump launch left a vertex short of its root
  uint32_t jdummy;  // flag word of the earlier jump launches (not read)
  uint32_t iter;  // body executions (two rounds each)
  uint32_t reason, slot;
};
void launch_round_init(GraphRounds *g, uint64_t m, uint64_t n_act, cudaStream_t s);
// The same from a device count of edges (at most cap); the active count is
// zeroed for the hooking launch of the call's first round to fill.
void launch_round_init_dev(GraphRounds *g, const u64 *m_dev, uint64_t cap, cudaStream_t s);
// The graph's first node: enter the loop only with active vertices and edges
// and a finished jump (else end it; a jump left short is ERR_HANDBACK in
// *err_handback when that is given, the device-driven mode).
void launch_round_pre(GraphRounds *g, cudaGraphConditionalHandle h, u64 *out_counts, uint32_t *err_handback,
                      cudaStream_t s);
void launch_round_check(GraphRounds *g, int base_ok, uint32_t *err_handback, cudaStream_t s);
void launch_round_cond(GraphRounds *g, cudaGraphConditionalHandle h, int base_ok, uint32_t max_iter, u64 *out_counts,
                       uint32_t *err_handback, cudaStream_t s);

// single-block base case: the last rounds of a Borůvka call in one launch
constexpr uint32_t BASE_MAX_N = 4096;  // live components (16-bit local ends; shared-memory vertex arrays)
constexpr uint64_t BASE_MAX_M = 6144;  // live edges (fit the tile kernel's shared-memory edge capacity)
struct BaseScratch {
  uint32_t *loc;      // [n] local index of each live component (only those entries are written)
  uint32_t *ends;     // [m] packed local ends
  u64 *cutmin;        // [BASE_MAX_N] all ones (no cut limit)
  u64 *offsets;       // [2]
  uint32_t *plocal;   // [BASE_MAX_N] local root of each live component
  EdgeOut rest;       // [m] edges left between final components (discarded)
  u64 *rest_fill;
};
// False (nothing launched) when the call does not fit the base case.
bool launch_base_case(const uint32_t *act, uint32_t n_act, EdgeList cur, uint64_t m, uint32_t *parent, uint32_t *bits,
                      const BaseScratch &b, uint32_t *err, cudaStream_t s, int filter_heavy, u64 *wsum);
void launch_iota(uint32_t *p, uint64_t n, int sms, cudaStream_t s);

}  // namespace mstgpu
