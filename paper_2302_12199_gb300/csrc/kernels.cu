// CUDA kernels of the Borůvka round and of Filter-Borůvka, for sm_103a.
//
// Everything here is integer work on edge lists stored as SoA uint32 arrays
// (u, v, w, id).  The order on edges is the uint64 key (w << 32) | id, a strict
// total order (paper Section 2.3: ties broken consistently so that the MST is
// unique).  Inside one list the ids ascend with the position ("slot"), so the
// solver keys edges by (w << 32) | slot, which orders them exactly as
// (w << 32) | id while letting a vertex find its chosen edge by slot.
//
// Stream compaction (relabel, partition, filter, dedupe, active vertices,
// output ids) is one pass per list: each 256-thread block takes the next tile
// of 2048 items from a dynamic counter, scans its keep flags, and learns the
// tile's output offset by a decoupled look-back over the preceding tiles' status
// words (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016).  Survivors keep their input order.  Every wait is bounded.
#include <cstdint>

#include "internal.h"

namespace mstgpu {

constexpr int BLOCK = 256;
constexpr int ITEMS = 8;
constexpr int TILE = BLOCK * ITEMS;
constexpr uint32_t SPIN_LIMIT = 1u << 21;  // look-back polls before giving up (about a second)
constexpr uint32_t JUMP_STEPS = 64;        // pointer steps per jump launch
constexpr u64 PAIR_EMPTY = ~0ULL;

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ u64 ld_relaxed(const u64 *p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(u64 *p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void load8(const uint32_t *p, uint64_t base, uint32_t (&x)[ITEMS]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p + base);
  const uint4 a = __ldg(q), b = __ldg(q + 1);
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

__device__ __forceinline__ u64 edge_key(uint32_t w, uint64_t slot) { return ((u64)w << 32) | (u64)(uint32_t)slot; }

__device__ __forceinline__ u64 pair_of(uint32_t a, uint32_t b) {
  return a < b ? (((u64)a << 32) | b) : (((u64)b << 32) | a);
}

__device__ __forceinline__ u64 mix64(u64 z) {  // splitmix64 finaliser
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Output #i of the splitmix64 sequence whose state starts at `state`
// (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ u64 splitmix64_at(u64 state, u64 i) {
  return mix64(state + (i + 1ULL) * 0x9e3779b97f4a7c15ULL);
}

// Exclusive block-wide scan of one uint32 per thread (BLOCK threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t &total, uint32_t *s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const uint32_t wv = lane < BLOCK / 32 ? s_warp[lane] : 0u;
    uint32_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < BLOCK / 32) s_warp[lane] = wi - wv;
    if (lane == BLOCK / 32 - 1) s_warp[BLOCK / 32] = wi;
  }
  __syncthreads();
  total = s_warp[BLOCK / 32];
  return s_warp[wid] + incl - x;
}

// Decoupled look-back, run by all 32 lanes of warp 0.  Publishes the tile's
// aggregate, waits (bounded) for predecessors, publishes the inclusive prefix
// and returns the tile's exclusive prefix.  Status word layout:
// epoch (bits 63..34) | flag (33..32: 1 aggregate, 2 inclusive, 3 error) | value.
__device__ uint32_t decoupled_lookback(const ScanState &st, uint32_t tile, uint32_t aggregate, bool &error) {
  const uint32_t lane = threadIdx.x & 31;
  const u64 tag = (u64)st.epoch << 34;
  error = false;
  if (tile == 0) {
    if (lane == 0) st_relaxed(&st.status[0], tag | (2ULL << 32) | aggregate);
    return 0;
  }
  if (lane == 0) st_relaxed(&st.status[tile], tag | (1ULL << 32) | aggregate);
  uint32_t exclusive = 0, spins = 0;
  long long pred = (long long)tile - 1 - (long long)lane;
  for (;;) {
    u64 s = 0;
    uint32_t flag = 2;
    for (;;) {
      if (pred >= 0) {
        s = ld_relaxed(&st.status[pred]);
        flag = ((uint32_t)(s >> 34) == st.epoch) ? (uint32_t)((s >> 32) & 3u) : 0u;
      } else {
        s = 0;
        flag = 2;
      }
      if (__all_sync(0xffffffffu, flag != 0)) break;
      if (++spins > SPIN_LIMIT) {
        error = true;
        break;
      }
      __nanosleep(64);
    }
    if (error || __any_sync(0xffffffffu, flag == 3)) {
      error = true;
      break;
    }
    const uint32_t incl = __ballot_sync(0xffffffffu, flag == 2);
    const int first = incl ? __ffs(incl) - 1 : 32;
    uint32_t val = (int)lane <= first ? (uint32_t)(s & 0xffffffffULL) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    exclusive += val;
    if (incl) break;
    pred -= 32;
  }
  if (lane == 0) {
    if (error)
      st_relaxed(&st.status[tile], tag | (3ULL << 32));
    else
      st_relaxed(&st.status[tile], tag | (2ULL << 32) | (u64)(exclusive + aggregate));
  }
  return exclusive;
}

// Tile bookkeeping shared by the scan kernels.  Returns false when this block
// has no tile (more blocks than tiles).
struct TileInfo {
  uint32_t tile, ntiles;
};

__device__ __forceinline__ bool acquire_tile(const ScanState &st, uint64_t count, uint32_t *s_tile, TileInfo &t) {
  t.ntiles = (uint32_t)((count + TILE - 1) / TILE);
  if (threadIdx.x == 0) *s_tile = atomicAdd(&st.tile_ctr[st.epoch & 1u], 1u);
  __syncthreads();
  t.tile = *s_tile;
  if (t.tile >= t.ntiles) {
    if (t.ntiles == 0 && t.tile == 0 && threadIdx.x == 0) {
      *st.total = 0;
      st.tile_ctr[(st.epoch + 1) & 1u] = 0;
    }
    return false;
  }
  return true;
}

// Scan + look-back for one tile.  Returns the tile's output offset; false on a
// look-back error (the tile then writes nothing).
__device__ __forceinline__ bool tile_offsets(const ScanState &st, const TileInfo &t, uint32_t count,
                                             uint32_t &thread_excl, uint32_t &tile_total, uint64_t &tile_base,
                                             uint32_t *s_warp, uint32_t *s_excl, uint32_t *s_err) {
  thread_excl = block_exclusive_scan(count, tile_total, s_warp);
  if (threadIdx.x < 32) {
    bool err;
    const uint32_t ex = decoupled_lookback(st, t.tile, tile_total, err);
    if (threadIdx.x == 0) {
      *s_excl = ex;
      *s_err = err ? 1u : 0u;
    }
  }
  __syncthreads();
  if (*s_err) {
    if (threadIdx.x == 0) atomicOr(st.err, ERR_LOOKBACK);
    return false;
  }
  tile_base = *s_excl;
  if (t.tile == t.ntiles - 1 && threadIdx.x == 0) {
    *st.total = tile_base + tile_total;
    st.tile_ctr[(st.epoch + 1) & 1u] = 0;  // the next launch uses the other counter
  }
  return true;
}

// best[c] = min(best[c], key) for up to 2*ITEMS (vertex, key) pairs.  The
// current value is read first (from L2) and the atomic is skipped when it
// cannot lower it; the atomic's result is unused, so it compiles to a reduction.
__device__ __forceinline__ void relax_pairs(u64 *best, const uint32_t (&a)[ITEMS], const uint32_t (&b)[ITEMS],
                                            const u64 (&key)[ITEMS], uint32_t mask) {
  u64 ca[ITEMS], cb[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    ca[k] = (mask >> k & 1) ? __ldcg(best + a[k]) : 0ULL;
    cb[k] = (mask >> k & 1) ? __ldcg(best + b[k]) : 0ULL;
  }
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    if (key[k] < ca[k]) atomicMin(best + a[k], key[k]);
    if (key[k] < cb[k]) atomicMin(best + b[k], key[k]);
  }
}

__device__ __forceinline__ bool hash_insert(HashSlot *t, uint64_t mask, u64 pair, u64 key) {
  uint64_t h = mix64(pair) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    u64 cur = __ldcg(&t[h].pair);
    if (cur == PAIR_EMPTY) {
      cur = atomicCAS(&t[h].pair, PAIR_EMPTY, pair);
      if (cur == PAIR_EMPTY) cur = pair;
    }
    if (cur == pair) {
      if (key < __ldcg(&t[h].key)) atomicMin(&t[h].key, key);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

__device__ __forceinline__ u64 hash_lookup(const HashSlot *t, uint64_t mask, u64 pair) {
  uint64_t h = mix64(pair) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const u64 cur = __ldg(&t[h].pair);
    if (cur == pair) return __ldg(&t[h].key);
    if (cur == PAIR_EMPTY) return KEY_INF;
    h = (h + 1) & mask;
  }
  return KEY_INF;
}

// ---------------------------------------------------------------- compaction

// One stream-compaction pass over an edge list; see CompactMode.  Survivors
// keep their order.  Optional post actions with the survivors' output slots:
// relax best[] (minEdges of the next round, fused) and/or insert the pair into
// the dedupe hash table.
template <int MODE, bool VEC>
__global__ void __launch_bounds__(BLOCK) compact_kernel(CompactArgs a) {
  __shared__ uint32_t s_u[TILE], s_v[TILE], s_w[TILE], s_id[TILE];
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  __shared__ uint32_t s_tile, s_excl, s_err;

  const uint64_t m = a.m_dev ? *a.m_dev : a.m;
  TileInfo t;
  if (!acquire_tile(a.st, m, &s_tile, t)) return;
  const uint64_t base = (uint64_t)t.tile * TILE + (uint64_t)threadIdx.x * ITEMS;

  uint32_t eu[ITEMS], ev[ITEMS], ew[ITEMS], ei[ITEMS];
  if (VEC && base + ITEMS <= m) {
    load8(a.in.u, base, eu);
    load8(a.in.v, base, ev);
    load8(a.in.w, base, ew);
    if (a.in.id) {
      load8(a.in.id, base, ei);
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) ei[k] = (uint32_t)(base + k);
    }
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint64_t j = base + k;
      if (j < m) {
        eu[k] = __ldg(a.in.u + j);
        ev[k] = __ldg(a.in.v + j);
        ew[k] = __ldg(a.in.w + j);
        ei[k] = a.in.id ? __ldg(a.in.id + j) : (uint32_t)j;
      } else {
        eu[k] = ev[k] = ew[k] = ei[k] = 0;
      }
    }
  }

  u64 pivot = 0;
  if (MODE == CM_PARTITION || MODE == CM_FILTER) pivot = a.pivot_dev ? *a.pivot_dev : a.pivot;

  uint32_t keep = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint64_t j = base + k;
    bool ok = j < m;
    if (ok && a.validate && (eu[k] >= a.n || ev[k] >= a.n)) {
      atomicOr(a.st.err, ERR_VERTEX);
      ok = false;
    }
    if (MODE == CM_RELABEL) {
      if (ok) {
        eu[k] = __ldg(a.label + eu[k]);
        ev[k] = __ldg(a.label + ev[k]);
        ok = eu[k] != ev[k];
      }
    } else if (MODE == CM_PARTITION) {
      ok = ok && eu[k] != ev[k] && (((u64)ew[k] << 32) | ei[k]) <= pivot;
    } else if (MODE == CM_FILTER) {
      if (ok && (((u64)ew[k] << 32) | ei[k]) > pivot) {
        eu[k] = __ldg(a.label + eu[k]);
        ev[k] = __ldg(a.label + ev[k]);
        ok = eu[k] != ev[k];
      } else {
        ok = false;
      }
    } else {  // CM_DEDUPE
      if (ok) ok = hash_lookup(a.table, a.tmask, pair_of(eu[k], ev[k])) == edge_key(ew[k], j);
    }
    keep |= (ok ? 1u : 0u) << k;
  }

  uint32_t excl, total;
  uint64_t obase;
  if (!tile_offsets(a.st, t, __popc(keep), excl, total, obase, s_warp, &s_excl, &s_err)) return;

  uint32_t lp = excl;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    if (keep >> k & 1) {
      s_u[lp] = eu[k];
      s_v[lp] = ev[k];
      s_w[lp] = ew[k];
      s_id[lp] = ei[k];
      ++lp;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < total; i += BLOCK) {
    a.out.u[obase + i] = s_u[i];
    a.out.v[obase + i] = s_v[i];
    a.out.w[obase + i] = s_w[i];
    a.out.id[obase + i] = s_id[i];
  }

  if (a.best || a.hash_insert) {
    u64 key[ITEMS];
    lp = excl;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      key[k] = edge_key(ew[k], obase + lp);
      lp += keep >> k & 1;
    }
    if (a.best) relax_pairs(a.best, eu, ev, key, keep);
    if (a.hash_insert) {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k)
        if ((keep >> k & 1) && !hash_insert(a.table, a.tmask, pair_of(eu[k], ev[k]), key[k]))
          atomicOr(a.st.err, ERR_HASH);
    }
  }
}

// --------------------------------------------------------------- min edges

// minEdges of a round that starts from a stored list (the input, or a list
// built by partition/filter): best[c] = min slot key over incident edges.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK) min_edges_kernel(EdgeList in, uint64_t m, uint32_t n, int validate,
                                                          u64 *best, uint32_t *err) {
  const uint64_t nchunks = (m + ITEMS - 1) / ITEMS;
  for (uint64_t ch = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; ch < nchunks; ch += (uint64_t)gridDim.x * BLOCK) {
    const uint64_t base = ch * ITEMS;
    uint32_t eu[ITEMS], ev[ITEMS], ew[ITEMS];
    if (VEC && base + ITEMS <= m) {
      load8(in.u, base, eu);
      load8(in.v, base, ev);
      load8(in.w, base, ew);
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const uint64_t j = base + k;
        eu[k] = j < m ? __ldg(in.u + j) : 0u;
        ev[k] = j < m ? __ldg(in.v + j) : 0u;
        ew[k] = j < m ? __ldg(in.w + j) : 0u;
      }
    }
    uint32_t mask = 0;
    u64 key[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      bool ok = base + k < m;
      if (ok && validate && (eu[k] >= n || ev[k] >= n)) {
        atomicOr(err, ERR_VERTEX);
        ok = false;
      }
      ok = ok && eu[k] != ev[k];
      mask |= (ok ? 1u : 0u) << k;
      key[k] = edge_key(ew[k], base + k);
    }
    relax_pairs(best, eu, ev, key, mask);
  }
}

// -------------------------------------------------------------------- hook

// Hooking (Section 2.3 / 4.2) over the candidate vertices: a vertex c with
// best[c] != INF points to the other end of its minimum edge; in a 2-cycle
// (both ends chose the same edge) the smaller vertex stays root.  Each chosen
// edge's id is set once in the bitmap (by the vertex that is not the root).
// The active vertices (best != INF) are compacted, in order, into active_out.
template <bool IOTA>
__global__ void __launch_bounds__(BLOCK) hook_kernel(HookArgs a) {
  __shared__ uint32_t s_c[TILE];
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  __shared__ uint32_t s_tile, s_excl, s_err;

  const uint64_t nc = a.ncand_dev ? *a.ncand_dev : a.ncand;
  TileInfo t;
  if (!acquire_tile(a.st, nc, &s_tile, t)) return;
  const uint64_t base = (uint64_t)t.tile * TILE + (uint64_t)threadIdx.x * ITEMS;

  uint32_t c[ITEMS];
  u64 kk[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint64_t j = base + k;
    c[k] = 0;
    kk[k] = KEY_INF;
    if (j < nc) {
      c[k] = IOTA ? (uint32_t)j : __ldg(a.cand + j);
      kk[k] = a.best[c[k]];
    }
  }
  uint32_t keep = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    if (kk[k] == KEY_INF) continue;
    keep |= 1u << k;
    const uint32_t slot = (uint32_t)kk[k];
    const uint32_t x = __ldg(a.list.u + slot), y = __ldg(a.list.v + slot);
    const uint32_t other = x ^ y ^ c[k];
    const bool root = a.best[other] == kk[k] && c[k] < other;
    a.parent[c[k]] = root ? c[k] : other;
    if (!root) {
      const uint32_t id = a.list.id ? __ldg(a.list.id + slot) : slot;
      atomicOr(a.chosen_bits + (id >> 5), 1u << (id & 31));
    }
  }

  uint32_t excl, total;
  uint64_t obase;
  if (!tile_offsets(a.st, t, __popc(keep), excl, total, obase, s_warp, &s_excl, &s_err)) return;
  uint32_t lp = excl;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k)
    if (keep >> k & 1) s_c[lp++] = c[k];
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < total; i += BLOCK) a.active_out[obase + i] = s_c[i];
}

// --------------------------------------------------------- pointer jumping

// Pointer doubling toward the roots (Section 4.2): each listed vertex follows
// parent pointers (reading the other threads' progress) for at most JUMP_STEPS
// steps and stores the furthest ancestor reached; `flag` is set if some vertex
// did not reach its root, and the host launches again.  Parent values only ever
// move toward the root, so concurrent reads and writes are benign.  When
// reset_best is set, best[c] is returned to INF for the next round.
__global__ void __launch_bounds__(BLOCK) jump_kernel(const uint32_t *act, const u64 *count_dev, uint64_t count_host,
                                                     uint32_t *parent, u64 *best, int reset_best, uint32_t *flag) {
  const uint64_t cnt = count_dev ? *count_dev : count_host;
  for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * BLOCK) {
    const uint32_t c = act ? __ldg(act + i) : (uint32_t)i;
    if (reset_best) best[c] = KEY_INF;
    uint32_t p = __ldcg(parent + c);
    uint32_t steps = 0;
    bool done = false;
    while (steps < JUMP_STEPS) {
      const uint32_t pp = __ldcg(parent + p);
      if (pp == p) {
        done = true;
        break;
      }
      p = pp;
      ++steps;
    }
    if (!done) atomicOr(flag, 1u);
    if (steps > 0) __stcg(parent + c, p);
  }
}

// ------------------------------------------------------------- small kernels

__global__ void hash_insert_kernel(EdgeList in, uint64_t m, HashSlot *table, uint64_t tmask, uint32_t *err) {
  for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < m; j += (uint64_t)gridDim.x * BLOCK) {
    const uint32_t u = in.u[j], v = in.v[j];
    if (u == v) continue;
    if (!hash_insert(table, tmask, pair_of(u, v), edge_key(in.w[j], j))) atomicOr(err, ERR_HASH);
  }
}

__global__ void best_slot_to_id_kernel(u64 *best, uint32_t n, const uint32_t *ids) {
  for (uint64_t c = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; c < n; c += (uint64_t)gridDim.x * BLOCK) {
    const u64 k = best[c];
    if (k != KEY_INF) best[c] = (k & 0xffffffff00000000ULL) | ids[(uint32_t)k];
  }
}

__global__ void iota_kernel(uint32_t *p, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (uint64_t)gridDim.x * BLOCK)
    p[i] = (uint32_t)i;
}

__global__ void u64_to_u32_kernel(const u64 *src, uint32_t *dst) { *dst = (uint32_t)*src; }

// ------------------------------------------------------------------ pivot

// PivotSelection (Alg. 2): sample k is the edge at position
// floor(splitmix64_at(state, k) * m / 2^64); its key is stored.
__global__ void pivot_sample_kernel(EdgeList in, uint64_t m_host, const u64 *m_dev, u64 state, uint32_t sample,
                                    u64 *out) {
  const uint64_t m = m_dev ? *m_dev : m_host;
  for (uint32_t i = blockIdx.x * BLOCK + threadIdx.x; i < sample; i += gridDim.x * BLOCK) {
    if (m == 0) {
      out[i] = KEY_INF;
      continue;
    }
    const uint64_t j = __umul64hi(splitmix64_at(state, i), m);
    out[i] = ((u64)__ldg(in.w + j) << 32) | (u64)(in.id ? __ldg(in.id + j) : (uint32_t)j);
  }
}

// The sample key of rank sample/2, by radix selection in one block: bytes are
// fixed from the most significant one that differs between the sample's
// minimum and maximum, using a 256-bin histogram per byte.
constexpr int SEL_THREADS = 1024;
__global__ void __launch_bounds__(SEL_THREADS) pivot_select_kernel(const u64 *keys, uint32_t sample, u64 *out) {
  __shared__ uint32_t hist[256];
  __shared__ u64 s_red[2][SEL_THREADS / 32];
  __shared__ u64 s_prefix, s_mask;
  __shared__ uint32_t s_rank;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  u64 mn = KEY_INF, mx = 0;
  for (uint32_t i = threadIdx.x; i < sample; i += SEL_THREADS) {
    const u64 k = keys[i];
    mn = k < mn ? k : mn;
    mx = k > mx ? k : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u64 a = __shfl_xor_sync(0xffffffffu, mn, o), b = __shfl_xor_sync(0xffffffffu, mx, o);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if (lane == 0) {
    s_red[0][wid] = mn;
    s_red[1][wid] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < SEL_THREADS / 32; ++i) {
      mn = s_red[0][i] < mn ? s_red[0][i] : mn;
      mx = s_red[1][i] > mx ? s_red[1][i] : mx;
    }
    s_red[0][0] = mn;
    s_red[1][0] = mx;
  }
  __syncthreads();
  mn = s_red[0][0];
  mx = s_red[1][0];
  if (mn == mx || sample == 0) {
    if (threadIdx.x == 0) *out = mn;
    return;
  }
  const int hb = 63 - __clzll((long long)(mn ^ mx));
  const int start = (hb / 8) * 8;
  if (threadIdx.x == 0) {
    s_mask = start + 8 >= 64 ? 0ULL : ~((1ULL << (start + 8)) - 1ULL);
    s_prefix = mn & s_mask;
    s_rank = sample / 2;
  }
  const uint32_t iters = (sample + SEL_THREADS - 1) / SEL_THREADS;
  for (int shift = start; shift >= 0; shift -= 8) {
    if (threadIdx.x < 256) hist[threadIdx.x] = 0;
    __syncthreads();
    const u64 prefix = s_prefix, mask = s_mask;
    for (uint32_t it = 0; it < iters; ++it) {
      const uint32_t i = it * SEL_THREADS + threadIdx.x;
      uint32_t d = 256;
      if (i < sample) {
        const u64 k = keys[i];
        if ((k & mask) == prefix) d = (uint32_t)(k >> shift) & 255u;
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (d < 256 && lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (wid == 0) {
      uint32_t sum = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) sum += hist[lane * 8 + b];
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t rank = s_rank;
      const uint32_t hit = __ballot_sync(0xffffffffu, incl > rank);
      if (lane == __ffs(hit) - 1) {
        uint32_t below = incl - sum;
        int d = lane * 8;
        while (below + hist[d] <= rank) below += hist[d++];
        s_prefix = prefix | ((u64)d << shift);
        s_mask = mask | (0xffULL << shift);
        s_rank = rank - below;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s_prefix;
}

// ---------------------------------------------------------------- finalize

// Output (Section 2.2; edge ids, Section 6.2): set bits of the chosen-edge
// bitmap become ascending ids; their weights are summed into a uint64.
__global__ void __launch_bounds__(BLOCK) finalize_kernel(const uint32_t *bits, uint64_t nwords, const uint32_t *w,
                                                         uint32_t *out_ids, uint32_t *out_count, u64 *total_weight,
                                                         ScanState st) {
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  __shared__ u64 s_sum[BLOCK / 32];
  __shared__ uint32_t s_tile, s_excl, s_err;
  TileInfo t;
  if (!acquire_tile(st, nwords, &s_tile, t)) {
    if (t.ntiles == 0 && t.tile == 0 && threadIdx.x == 0) *out_count = 0;
    return;
  }
  const uint64_t base = (uint64_t)t.tile * TILE + (uint64_t)threadIdx.x * ITEMS;
  uint32_t wd[ITEMS], cnt = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    wd[k] = base + k < nwords ? bits[base + k] : 0u;
    cnt += __popc(wd[k]);
  }
  uint32_t excl, total;
  uint64_t obase;
  if (!tile_offsets(st, t, cnt, excl, total, obase, s_warp, &s_excl, &s_err)) return;
  uint64_t pos = obase + excl;
  u64 wsum = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    uint32_t word = wd[k];
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      const uint32_t id = (uint32_t)((base + k) * 32 + b);
      out_ids[pos++] = id;
      wsum += __ldg(w + id);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 s = 0;
    for (int i = 0; i < BLOCK / 32; ++i) s += s_sum[i];
    if (s) atomicAdd(total_weight, s);
    if (t.tile == t.ntiles - 1) *out_count = (uint32_t)(obase + total);
  }
}

// ---------------------------------------------------------------- launchers

static inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static inline unsigned grid_for(uint64_t items_per_block_units, int sms, int per_sm) {
  const uint64_t cap = (uint64_t)(sms > 0 ? sms : 152) * (uint64_t)per_sm;
  uint64_t g = items_per_block_units;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

int max_scan_tiles(uint64_t count) { return (int)((count + TILE - 1) / TILE); }

template <int MODE>
static void launch_compact_mode(const CompactArgs &a, unsigned grid, cudaStream_t s) {
  const bool vec = aligned16(a.in.u) && aligned16(a.in.v) && aligned16(a.in.w) && (!a.in.id || aligned16(a.in.id));
  if (vec)
    compact_kernel<MODE, true><<<grid, BLOCK, 0, s>>>(a);
  else
    compact_kernel<MODE, false><<<grid, BLOCK, 0, s>>>(a);
}

void launch_compact(CompactMode mode, const CompactArgs &a, uint64_t max_count, cudaStream_t s) {
  const unsigned grid = (unsigned)(max_scan_tiles(max_count) > 0 ? max_scan_tiles(max_count) : 1);
  switch (mode) {
    case CM_RELABEL: launch_compact_mode<CM_RELABEL>(a, grid, s); break;
    case CM_PARTITION: launch_compact_mode<CM_PARTITION>(a, grid, s); break;
    case CM_FILTER: launch_compact_mode<CM_FILTER>(a, grid, s); break;
    case CM_DEDUPE: launch_compact_mode<CM_DEDUPE>(a, grid, s); break;
  }
}

void launch_min_edges(EdgeList in, uint64_t m, uint32_t n, int validate, u64 *best, uint32_t *err, int sms,
                      cudaStream_t s) {
  if (m == 0) return;
  const unsigned grid = grid_for((m + (uint64_t)TILE - 1) / TILE, sms, 8);
  if (aligned16(in.u) && aligned16(in.v) && aligned16(in.w))
    min_edges_kernel<true><<<grid, BLOCK, 0, s>>>(in, m, n, validate, best, err);
  else
    min_edges_kernel<false><<<grid, BLOCK, 0, s>>>(in, m, n, validate, best, err);
}

void launch_hook(const HookArgs &a, uint64_t max_cand, cudaStream_t s) {
  const unsigned grid = (unsigned)(max_scan_tiles(max_cand) > 0 ? max_scan_tiles(max_cand) : 1);
  if (a.cand)
    hook_kernel<false><<<grid, BLOCK, 0, s>>>(a);
  else
    hook_kernel<true><<<grid, BLOCK, 0, s>>>(a);
}

void launch_jump(const uint32_t *act, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                 uint32_t *parent, u64 *best, int reset_best, uint32_t *flag, int sms, cudaStream_t s) {
  if (max_count == 0) return;
  const unsigned grid = grid_for((max_count + BLOCK - 1) / BLOCK, sms, 8);
  jump_kernel<<<grid, BLOCK, 0, s>>>(act, count_dev, count_host, parent, best, reset_best, flag);
}

void launch_hash_insert(EdgeList in, uint64_t m, HashSlot *table, uint64_t tmask, uint32_t *err, int sms,
                        cudaStream_t s) {
  if (m == 0) return;
  hash_insert_kernel<<<grid_for((m + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(in, m, table, tmask, err);
}

void launch_best_slot_to_id(u64 *best, uint32_t n, const uint32_t *ids, int sms, cudaStream_t s) {
  if (n == 0 || ids == nullptr) return;
  best_slot_to_id_kernel<<<grid_for(((uint64_t)n + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(best, n, ids);
}

void launch_pivot(EdgeList in, uint64_t m, const u64 *m_dev, u64 state, uint32_t sample, u64 *sample_buf,
                  u64 *pivot_out, cudaStream_t s) {
  const unsigned g = (sample + BLOCK - 1) / BLOCK;
  pivot_sample_kernel<<<g > 0 ? g : 1, BLOCK, 0, s>>>(in, m, m_dev, state, sample, sample_buf);
  pivot_select_kernel<<<1, SEL_THREADS, 0, s>>>(sample_buf, sample, pivot_out);
}

void launch_finalize(const uint32_t *bits, uint64_t m, const uint32_t *w, uint32_t *out_ids, uint32_t *out_count,
                     u64 *total_weight, ScanState st, cudaStream_t s) {
  const uint64_t nwords = (m + 31) / 32;
  const unsigned grid = (unsigned)(max_scan_tiles(nwords) > 0 ? max_scan_tiles(nwords) : 1);
  finalize_kernel<<<grid, BLOCK, 0, s>>>(bits, nwords, w, out_ids, out_count, total_weight, st);
}

void launch_iota(uint32_t *p, uint64_t n, int sms, cudaStream_t s) {
  if (n == 0) return;
  iota_kernel<<<grid_for((n + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(p, n);
}

void launch_u64_to_u32(const u64 *src, uint32_t *dst, cudaStream_t s) { u64_to_u32_kernel<<<1, 1, 0, s>>>(src, dst); }

}  // namespace mstgpu
