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
};

// Small per-handle device state.
struct DevState {
  uint32_t err;
  uint32_t jump_flag;   // set when a pointer-jump launch left a vertex short of its root
  uint32_t tile_ctr[2]; // dynamic tile counters of the scan kernels (alternating by epoch)
  u64 count[6];         // counts written by the last tile of a scan kernel
  u64 pivot;            // result of the pivot selection
};
enum { CNT_EDGES = 0, CNT_ACTIVE = 1, CNT_TMP = 2, CNT_AUX = 3, CNT_USER = 4 };

// State of one decoupled look-back scan launch.
struct ScanState {
  u64 *status;       // one status word per tile: epoch(30) | flag(2) | value(32)
  uint32_t *tile_ctr;
  uint32_t epoch;    // 1 .. 2^30-1, different for every launch
  u64 *total;        // receives the scan total (written by the last tile)
  uint32_t *err;
};

struct HashSlot {
  u64 pair;  // (min(u,v) << 32) | max(u,v); all ones = empty
  u64 key;   // minimum (w << 32) | slot seen for this pair
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
  CM_DEDUPE = 3,     // keep iff the hash table holds this edge's slot key for its pair
};

struct CompactArgs {
  EdgeList in;
  uint64_t m;              // input length (used when m_dev == nullptr)
  const u64 *m_dev;        // input length in device memory, or nullptr
  EdgeOut out;
  const uint32_t *label;   // relabel / filter
  u64 pivot;               // partition / filter (used when pivot_dev == nullptr)
  const u64 *pivot_dev;
  u64 *best;               // if set: relax best[] with the output slot keys
  HashSlot *table;         // dedupe lookup, or insert target when hash_insert
  uint64_t tmask;
  int hash_insert;
  uint32_t n;              // vertex count, for validation
  int validate;            // check u, v < n (sets ERR_VERTEX, skips the edge)
  ScanState st;
};

struct HookArgs {
  const uint32_t *cand;    // candidate vertices; nullptr = 0..ncand-1
  uint64_t ncand;
  const u64 *ncand_dev;    // candidate count in device memory, or nullptr
  u64 *best;
  EdgeList list;           // the list whose slots the keys in best[] refer to
  uint32_t *parent;
  uint32_t *chosen_bits;   // bitmap over original edge ids
  uint32_t *active_out;    // compacted active vertices
  ScanState st;
};

// ---- launchers (kernels.cu); all asynchronous on `s` ----
int max_scan_tiles(uint64_t count);
void launch_compact(CompactMode mode, const CompactArgs &a, uint64_t max_count, cudaStream_t s);
void launch_min_edges(EdgeList in, uint64_t m, uint32_t n, int validate, u64 *best, uint32_t *err, int sms,
                      cudaStream_t s);
void launch_hook(const HookArgs &a, uint64_t max_cand, cudaStream_t s);
void launch_jump(const uint32_t *act, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                 uint32_t *parent, u64 *best, int reset_best, uint32_t *flag, int sms, cudaStream_t s);
void launch_hash_insert(EdgeList in, uint64_t m, HashSlot *table, uint64_t tmask, uint32_t *err, int sms,
                        cudaStream_t s);
void launch_best_slot_to_id(u64 *best, uint32_t n, const uint32_t *ids, int sms, cudaStream_t s);
void launch_pivot(EdgeList in, uint64_t m, const u64 *m_dev, u64 state, uint32_t sample, u64 *sample_buf,
                  u64 *pivot_out, cudaStream_t s);
void launch_finalize(const uint32_t *bits, uint64_t m, const uint32_t *w, uint32_t *out_ids, uint32_t *out_count,
                     u64 *total_weight, ScanState st, cudaStream_t s);
void launch_iota(uint32_t *p, uint64_t n, int sms, cudaStream_t s);
void launch_u64_to_u32(const u64 *src, uint32_t *dst, cudaStream_t s);

}  // namespace mstgpu
