// CUDA kernels of the Borůvka round and of Filter-Borůvka, for sm_103a.
//
// Everything here is integer work on edge lists stored as SoA uint32 arrays
// (u, v, w, id).  The order on edges is the uint64 key (w << 32) | id, a strict
// total order (paper Section 2.3: ties broken consistently so that the MST is
// unique); id is the edge's index in the caller's input.
//
// Stream compaction (relabel, partition, dedupe, active vertices) is one pass
// per list: each block takes a tile of B x I items (256 x 8 by default; the
// shape is a run-time choice), stages the tile's survivors in shared memory,
// and claims its output range with one atomic add.  The filter pass streams
// per warp instead (stream_warp_kernel).  Lists therefore come out in an
// unspecified order; nothing downstream depends on list order, because edges
// are keyed by id and a vertex finds its chosen edge through the input arrays.  The output ids (finalize) are the one
// ordered compaction: a decoupled look-back scan (Merrill & Garland, 2016).
// Every wait is bounded.
#include <algorithm>
#include <cstdint>

#include <cooperative_groups.h>

#include "internal.h"

namespace mstgpu {

constexpr int BLOCK = 256;
constexpr int ITEMS = 8;
constexpr int TILE = BLOCK * ITEMS;
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

// Striped item layout inside a tile of B * I items (B threads, I items each, I
// a multiple of 4): item k of thread t sits at tile offset
// (k / 4) * (B * 4) + 4 * t + k % 4.  Each warp-wide 16-byte load then covers
// 512 contiguous bytes (whole sectors, used once).  The defaults are the
// shape of the kernels that do not take one (BLOCK x ITEMS).
template <int B = BLOCK>
__device__ __forceinline__ uint32_t item_off(int k) {
  return (uint32_t)((k >> 2) * (B * 4) + 4 * threadIdx.x + (k & 3));
}

template <int B = BLOCK, int I = ITEMS>
__device__ __forceinline__ void load_striped(const uint32_t *p, uint64_t tile_base, uint32_t (&x)[I]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p + tile_base);
#pragma unroll
  for (int c = 0; c < I / 4; ++c) {
    const uint4 t = __ldg(q + c * B + threadIdx.x);
    x[4 * c] = t.x;
    x[4 * c + 1] = t.y;
    x[4 * c + 2] = t.z;
    x[4 * c + 3] = t.w;
  }
}

// Per-thread counts of kept items in the two chunks, packed for one scan.
__device__ __forceinline__ uint32_t packed_counts(uint32_t keep) {
  return (uint32_t)__popc(keep & 0xfu) | ((uint32_t)__popc(keep >> 4) << 16);
}

// Tile-local output position of kept item k, from the packed exclusive scan
// value of this thread and the packed tile total.
__device__ __forceinline__ uint32_t local_pos(uint32_t keep, int k, uint32_t excl_p, uint32_t total_p) {
  if (k < 4) return (excl_p & 0xffffu) + (uint32_t)__popc(keep & ((1u << k) - 1u));
  return (total_p & 0xffffu) + (excl_p >> 16) + (uint32_t)__popc((keep >> 4) & ((1u << (k - 4)) - 1u));
}

__device__ __forceinline__ u64 edge_key(uint32_t w, uint32_t id) { return ((u64)w << 32) | (u64)id; }

// Relaxation key of an edge as seen from one end (see KeyLayout).
__device__ __forceinline__ u64 relax_key(const KeyLayout &kl, uint32_t w, uint32_t id, uint32_t other) {
  return kl.packed ? (((u64)w << (kl.idbits + kl.vbits)) | ((u64)id << kl.vbits) | (u64)other) : edge_key(w, id);
}
__device__ __forceinline__ uint32_t key_edge_id(const KeyLayout &kl, u64 key) {
  return kl.packed ? (uint32_t)((key >> kl.vbits) & ((1ULL << kl.idbits) - 1)) : (uint32_t)key;
}
// Do two keys name the same edge (the 2-cycle test)?
__device__ __forceinline__ bool same_edge(const KeyLayout &kl, u64 a, u64 b) {
  return kl.packed ? (a >> kl.vbits) == (b >> kl.vbits) : a == b;
}

__device__ __forceinline__ bool aligned16_dev(const void *p) { return ((uintptr_t)p & 15u) == 0; }

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

// Exclusive block-wide scan of one uint32 per thread (B threads; s_warp holds
// B / 32 + 1 words).
template <int B = BLOCK>
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
    const uint32_t wv = lane < B / 32 ? s_warp[lane] : 0u;
    uint32_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < B / 32) s_warp[lane] = wi - wv;
    if (lane == B / 32 - 1) s_warp[B / 32] = wi;
  }
  __syncthreads();
  total = s_warp[B / 32];
  return s_warp[wid] + incl - x;
}

// Decoupled look-back by the whole block.  Publishes the tile's aggregate,
// then examines LB_WINDOW = BLOCK * LB_PER_THREAD predecessors per round (each
// thread polls LB_PER_THREAD status words, bounded), adds the values up to the
// nearest tile whose inclusive prefix is published, and continues further back
// only if none in the window has one; finally publishes its own inclusive
// prefix and returns the exclusive one.  A window as wide as the number of
// tiles in flight keeps the walk to one round.  Status word layout:
// epoch (bits 63..34) | flag (33..32: 1 aggregate, 2 inclusive, 3 error) | value.
constexpr int LB_PER_THREAD = 4;
constexpr int LB_WINDOW = BLOCK * LB_PER_THREAD;

struct LookbackShared {
  uint32_t first;    // smallest window offset holding an inclusive prefix
  uint32_t error;
  uint32_t sum[BLOCK / 32];
};

__device__ uint32_t decoupled_lookback(const ScanState &st, uint32_t tile, uint32_t aggregate, bool &error,
                                       LookbackShared &sh) {
  const u64 tag = (u64)st.epoch << 34;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (tile == 0) {
    if (threadIdx.x == 0) st_relaxed(&st.status[0], tag | (2ULL << 32) | aggregate);
    error = false;
    return 0;
  }
  if (threadIdx.x == 0) st_relaxed(&st.status[tile], tag | (1ULL << 32) | aggregate);
  uint32_t exclusive = 0;
  long long top = (long long)tile - 1;  // newest predecessor of the current window
  for (;;) {
    if (threadIdx.x == 0) {
      sh.first = LB_WINDOW;
      sh.error = 0;
    }
    __syncthreads();
    uint32_t val[LB_PER_THREAD], flag[LB_PER_THREAD];
#pragma unroll
    for (int k = 0; k < LB_PER_THREAD; ++k) {
      const long long pred = top - (long long)(k * BLOCK + threadIdx.x);  // window offset k*BLOCK+tid
      val[k] = 0;
      flag[k] = 2;
      if (pred >= 0) {
        uint32_t spins = 0;
        for (;;) {
          const u64 s = ld_relaxed(&st.status[pred]);
          flag[k] = ((uint32_t)(s >> 34) == st.epoch) ? (uint32_t)((s >> 32) & 3u) : 0u;
          val[k] = (uint32_t)s;
          if (flag[k] != 0) break;
          if (++spins >= st.spin_limit) {  // bounded: the predecessor never published
            flag[k] = 3;
            break;
          }
          __nanosleep(32);
        }
      }
      if (flag[k] == 3) atomicOr(&sh.error, 1u);
      if (flag[k] == 2) atomicMin(&sh.first, (uint32_t)(k * BLOCK + threadIdx.x));
    }
    __syncthreads();
    if (sh.error) {
      error = true;
      break;
    }
    const uint32_t first = sh.first;
    uint32_t part = 0;
#pragma unroll
    for (int k = 0; k < LB_PER_THREAD; ++k)
      if ((uint32_t)(k * BLOCK + threadIdx.x) <= first) part += val[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) sh.sum[wid] = part;
    __syncthreads();
    uint32_t win = 0;
#pragma unroll
    for (int i = 0; i < BLOCK / 32; ++i) win += sh.sum[i];
    exclusive += win;
    if (first < LB_WINDOW) {
      error = false;
      break;
    }
    top -= LB_WINDOW;
    __syncthreads();  // sh.sum is rewritten in the next round
  }
  if (threadIdx.x == 0) {
    if (error)
      st_relaxed(&st.status[tile], tag | (3ULL << 32));
    else
      st_relaxed(&st.status[tile], tag | (2ULL << 32) | (u64)(exclusive + aggregate));
  }
  return exclusive;
}

// Tile bookkeeping shared by the scan kernels.  Tile t is processed by block t
// (blocks are dispatched in index order, so every predecessor of a waiting
// block is already resident or finished).  Returns false when this block has
// no tile (the count is read on the device and the grid was sized for an upper
// bound).
struct TileInfo {
  uint32_t tile, ntiles;
};

__device__ __forceinline__ bool acquire_tile(const ScanState &st, uint64_t count, TileInfo &t) {
  t.ntiles = (uint32_t)((count + TILE - 1) / TILE);
  t.tile = blockIdx.x;
  if (t.tile >= t.ntiles) {
    if (t.ntiles == 0 && t.tile == 0 && threadIdx.x == 0) *st.total = 0;
    return false;
  }
  return true;
}

// Scan + look-back for one tile.  `packed` holds this thread's chunk-0 count in
// the low and chunk-1 count in the high 16 bits (each block total is at most
// TILE / 2, so the halves never carry).  Returns the packed exclusive scan, the
// packed tile total and the tile's output offset; false on a look-back error
// (the tile then writes nothing).
__device__ __forceinline__ bool tile_offsets(const ScanState &st, const TileInfo &t, uint32_t packed,
                                             uint32_t &excl_p, uint32_t &total_p, uint64_t &tile_base,
                                             uint32_t *s_warp, LookbackShared &sh) {
  excl_p = block_exclusive_scan(packed, total_p, s_warp);
  const uint32_t tile_total = (total_p & 0xffffu) + (total_p >> 16);
  bool err = false;
  const uint32_t ex = decoupled_lookback(st, t.tile, tile_total, err, sh);
  if (err) {
    if (threadIdx.x == 0) atomicOr(st.err, ERR_LOOKBACK);
    return false;
  }
  tile_base = ex;
  if (t.tile == t.ntiles - 1 && threadIdx.x == 0) *st.total = tile_base + tile_total;
  return true;
}

// Claims `total` output slots for this block's tile with one atomic add on the
// list's counter and broadcasts the base to the block (order of tiles in the
// output is unspecified; order inside a tile is kept).
__device__ __forceinline__ uint64_t tile_claim(unsigned long long *counter, uint32_t total, uint32_t *s_base) {
  if (threadIdx.x == 0) s_base[0] = total ? (uint32_t)atomicAdd(counter, (unsigned long long)total) : 0u;
  __syncthreads();
  return s_base[0];
}

// best[c] = min(best[c], key) for up to 2*ITEMS (vertex, key) pairs.  The
// current value is read first and the atomic is skipped when it cannot lower
// it.  The read may be served from L1 and be stale, which only costs an extra
// atomic (values only decrease); it keeps hub vertices from turning every edge
// into an L2 access.  The atomic's result is unused, so it is a reduction.
__device__ __forceinline__ void relax_pairs(u64 *best, const uint32_t (&a)[ITEMS], const uint32_t (&b)[ITEMS],
                                            const u64 (&key)[ITEMS], const u64 (&keyb)[ITEMS], uint32_t mask) {
  u64 ca[ITEMS], cb[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    ca[k] = (mask >> k & 1) ? __ldca(best + a[k]) : 0ULL;
    cb[k] = (mask >> k & 1) ? __ldca(best + b[k]) : 0ULL;
  }
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    if (key[k] < ca[k]) atomicMin(best + a[k], key[k]);
    if (keyb[k] < cb[k]) atomicMin(best + b[k], keyb[k]);
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

// Keep flags of a thread's ITEMS items for a compaction mode (see
// CompactMode); relabels eu/ev in place where the mode relabels.  Bit k =
// item k; only items whose bit is set in `valid` can be kept.
template <int MODE, int N>
__device__ __forceinline__ uint32_t keep_flags(const CompactArgs &a, uint32_t valid, u64 pivot, uint32_t (&eu)[N],
                                               uint32_t (&ev)[N], const uint32_t (&ew)[N], const uint32_t (&ei)[N],
                                               const uint32_t *gbits) {
  uint32_t keep = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    bool ok = (valid >> k) & 1u;
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
    } else if (MODE == CM_FILTER || MODE == CM_HEAVY) {
      ok = ok && (((u64)ew[k] << 32) | ei[k]) > pivot;  // heavy; resolved below for all items at once
    } else {  // CM_DEDUPE
      if (ok) ok = hash_lookup(a.table, a.tmask, pair_of(eu[k], ev[k])) == edge_key(ew[k], ei[k]);
    }
    keep |= (ok ? 1u : 0u) << k;
  }
  if (MODE == CM_HEAVY && gbits) {  // drop heavy edges inside the giant component; keep the ends
    uint32_t bu[N], bv[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const bool h = keep >> k & 1;
      bu[k] = h ? __ldg(gbits + (eu[k] >> 5)) : 0u;
      bv[k] = h ? __ldg(gbits + (ev[k] >> 5)) : 0u;
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
      if ((bu[k] >> (eu[k] & 31)) & (bv[k] >> (ev[k] & 31)) & 1u) keep &= ~(1u << k);
  }
  if (MODE == CM_FILTER) {
    // Heavy edges with both ends in the marked (largest) component lie inside
    // one component.  The bitmap words of all items are loaded together, then
    // the labels of the remaining items, so that each thread has one round of
    // independent loads in flight per step.
    if (gbits) {
      uint32_t bu[N], bv[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const bool h = keep >> k & 1;
        bu[k] = h ? __ldg(gbits + (eu[k] >> 5)) : 0u;
        bv[k] = h ? __ldg(gbits + (ev[k] >> 5)) : 0u;
      }
#pragma unroll
      for (int k = 0; k < N; ++k)
        if ((bu[k] >> (eu[k] & 31)) & (bv[k] >> (ev[k] & 31)) & 1u) keep &= ~(1u << k);
    }
    uint32_t lu[N], lv[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const bool h = keep >> k & 1;
      lu[k] = h ? __ldg(a.label + eu[k]) : 0u;
      lv[k] = h ? __ldg(a.label + ev[k]) : 0u;
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      eu[k] = lu[k];
      ev[k] = lv[k];
      if (lu[k] == lv[k]) keep &= ~(1u << k);
    }
  }
  return keep;
}

// Writes the kept items of a tile (B threads, I items each) to shared memory
// at their tile-local output positions (thread-major: thread t's kept items,
// in item order, follow those of threads 0..t-1; `excl` is the exclusive scan
// of the per-thread kept counts), stores them coalesced at obase, then runs
// the post actions on the survivors: relax best[] (the next round's minEdges,
// fused) and/or insert the pair into the dedupe hash table.
template <int B, int I>
__device__ __forceinline__ void emit_survivors(const CompactArgs &a, uint32_t keep, uint32_t excl, uint32_t total,
                                               uint64_t obase, const uint32_t (&eu)[I], const uint32_t (&ev)[I],
                                               const uint32_t (&ew)[I], const uint32_t (&ei)[I], uint32_t *s_u,
                                               uint32_t *s_v, uint32_t *s_w, uint32_t *s_id) {
#pragma unroll
  for (int k = 0; k < I; ++k) {
    if (keep >> k & 1) {
      const uint32_t lp = excl + (uint32_t)__popc(keep & ((1u << k) - 1u));
      s_u[lp] = eu[k];
      s_v[lp] = ev[k];
      s_w[lp] = ew[k];
      s_id[lp] = ei[k];
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < total; i += B) {
    a.out.u[obase + i] = s_u[i];
    a.out.v[obase + i] = s_v[i];
    a.out.w[obase + i] = s_w[i];
    a.out.id[obase + i] = s_id[i];
  }
  if (a.cur_u) {  // ends by id, for the hook of the round that relaxes this list
    for (uint32_t i = threadIdx.x; i < total; i += B) {
      a.cur_u[s_id[i]] = s_u[i];
      a.cur_v[s_id[i]] = s_v[i];
    }
  }
  // post actions read the survivors back from shared memory (coalesced; the
  // loaded edges' registers are dead by now)
  if (a.best) {
    for (uint32_t i0 = 0; i0 < total; i0 += 4 * B) {
      uint32_t x[4], y[4];
      u64 kx[4], ky[4], cx[4], cy[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t i = i0 + k * B + threadIdx.x;
        const bool ok = i < total;
        x[k] = ok ? s_u[i] : 0u;
        y[k] = ok ? s_v[i] : 0u;
        kx[k] = ok ? relax_key(a.kl, s_w[i], s_id[i], y[k]) : KEY_INF;
        ky[k] = ok ? relax_key(a.kl, s_w[i], s_id[i], x[k]) : KEY_INF;
        cx[k] = ok ? __ldca(a.best + x[k]) : 0ULL;
        cy[k] = ok ? __ldca(a.best + y[k]) : 0ULL;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (kx[k] < cx[k]) atomicMin(a.best + x[k], kx[k]);
        if (ky[k] < cy[k]) atomicMin(a.best + y[k], ky[k]);
      }
    }
  }
  if (a.hash_insert) {
    for (uint32_t i = threadIdx.x; i < total; i += B)
      if (!hash_insert(a.table, a.tmask, pair_of(s_u[i], s_v[i]), edge_key(s_w[i], s_id[i])))
        atomicOr(a.st.err, ERR_HASH);
  }
}

// The number of a tile's `total` survivors to write at obase: all of them, or
// those that fit below the output capacity (and ERR_OVERFLOW, once per tile).
// Writing the part that fits keeps every slot below the capacity written, so
// a reader that takes min(count, capacity) entries never sees an unwritten
// one.  The same in every thread of the block.
__device__ __forceinline__ uint32_t within_capacity(const CompactArgs &a, uint64_t obase, uint32_t total) {
  if (!a.out_cap || obase + total <= a.out_cap) return total;
  if (threadIdx.x == 0) atomicOr(a.st.err, ERR_OVERFLOW);
  return obase < a.out_cap ? (uint32_t)(a.out_cap - obase) : 0u;
}

__device__ __forceinline__ u64 compact_pivot(const CompactArgs &a, int mode) {
  return (mode == CM_PARTITION || mode == CM_FILTER || mode == CM_HEAVY) ? (a.pivot_dev ? *a.pivot_dev : a.pivot)
                                                                         : 0ULL;
}

// Bit k set iff item k of this thread's striped tile (base tb) is below m.
template <int B, int I>
__device__ __forceinline__ uint32_t valid_items_s(uint64_t tb, uint64_t m) {
  uint32_t valid = 0;
#pragma unroll
  for (int k = 0; k < I; ++k) valid |= (tb + item_off<B>(k) < m ? 1u : 0u) << k;
  return valid;
}

// Tile shapes the compaction and hook kernels are built for (threads per
// block B, items per thread I), chosen at run time (mst_config block_threads /
// items_per_thread).  Launch bounds come from a register budget per thread
// that each kernel needs at I items (measured with -Xptxas -v: the budgets
// below build without spills): resident blocks = 64K registers / (B x budget),
// at least 1 and at most 2048 threads.
template <int B, int I>
struct Shape {
  static constexpr int T = B * I;  // items per tile
  static constexpr int minb(int regs) {
    const int b = 65536 / (B * regs), cap = 2048 / B;
    return b < 1 ? 1 : (b > cap ? cap : b);
  }
  // budgets: the compaction, the persistent TMA compaction, the hook with and
  // without the far end packed in the key
  static constexpr int compact_regs = I <= 8 ? 64 : 128;
  static constexpr int tma_regs = I <= 4 ? 64 : (I <= 8 ? 80 : 128);
  static constexpr int hook_packed_regs = I <= 4 ? 32 : (I <= 8 ? 40 : 72);
  static constexpr int hook_regs = I <= 4 ? 64 : (I <= 8 ? 80 : 168);
};

// One stream-compaction pass over an edge list, one tile of B * I items per
// block; the staging buffer (16 bytes per item) is dynamic shared memory.
template <int MODE, bool VEC, int B, int I>
__global__ void __launch_bounds__(B, Shape<B, I>::minb(Shape<B, I>::compact_regs)) compact_kernel(CompactArgs a) {
  constexpr int T = Shape<B, I>::T;
  extern __shared__ __align__(16) uint32_t s_stage[];  // u, v, w, id: T each
  __shared__ uint32_t s_warp[B / 32 + 1];
  __shared__ uint32_t s_base[1];
  uint32_t *s_u = s_stage, *s_v = s_stage + T, *s_w = s_stage + 2 * T, *s_id = s_stage + 3 * T;

  const uint64_t m = a.m_dev ? min((uint64_t)*a.m_dev, a.m) : a.m;
  const uint64_t tb = (uint64_t)blockIdx.x * T;
  if (tb >= m) return;

  uint32_t eu[I], ev[I], ew[I], ei[I];
  if (VEC && tb + T <= m) {
    load_striped<B, I>(a.in.u, tb, eu);
    load_striped<B, I>(a.in.v, tb, ev);
    load_striped<B, I>(a.in.w, tb, ew);
    if (a.in.id) {
      load_striped<B, I>(a.in.id, tb, ei);
    } else {
#pragma unroll
      for (int k = 0; k < I; ++k) ei[k] = (uint32_t)(tb + item_off<B>(k));
    }
  } else {
#pragma unroll
    for (int k = 0; k < I; ++k) {
      const uint64_t j = tb + item_off<B>(k);
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
  const uint32_t valid = valid_items_s<B, I>(tb, m);
  const uint32_t keep = keep_flags<MODE>(a, valid, compact_pivot(a, MODE), eu, ev, ew, ei, a.giant_bits);
  if (a.max_w) {  // largest weight of the input, folded into this pass
    uint32_t mx = 0;
#pragma unroll
    for (int k = 0; k < I; ++k) mx = max(mx, (valid >> k & 1) ? ew[k] : 0u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > __ldca(a.max_w)) atomicMax(a.max_w, mx);  // rarely true after a few tiles
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<B>((uint32_t)__popc(keep), total, s_warp);
  const uint64_t obase = tile_claim(a.st.total, total, s_base);
  emit_survivors<B, I>(a, keep, excl, within_capacity(a, obase, total), obase, eu, ev, ew, ei, s_u, s_v, s_w, s_id);
}

// ------------------------------------------------ TMA-pipelined compaction

// The persistent form of compact_kernel for long lists: block b of G handles
// tiles b, b + G, b + 2G, ...  Full tiles arrive in a ring of TMA_STAGES
// shared-memory stages by bulk copies (cp.async.bulk, one per array, completion
// counted on the stage's mbarrier), issued TMA_STAGES tiles ahead; a stage is
// refilled as soon as its items are in registers.  So HBM keeps streaming the
// next tiles while the block waits on the current tile's label / bitmap
// gathers, scans it and stores it.  Blocks never wait for each other.
constexpr int TMA_STAGES = 1;
constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 24;

template <int T>
struct __align__(16) EdgeStage {
  uint32_t u[T], v[T], w[T], id[T];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64 *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u64 *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64 *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for phase `parity` of a stage barrier; false if it never came.
__device__ __forceinline__ bool mbar_wait_bounded(u64 *bar, uint32_t parity) {
  for (uint32_t i = 0; i < MBAR_SPIN_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, u64 *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Issues the bulk copies of full tile `tile` into stage `st` (one thread).
template <int T>
__device__ __forceinline__ void issue_tile(const CompactArgs &a, uint64_t tile, EdgeStage<T> *st, u64 *bar) {
  const uint32_t bytes = T * 4;
  const uint64_t off = tile * T;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order the stage's earlier generic reads
  mbar_arrive_expect_tx(bar, (a.in.id ? 4u : 3u) * bytes);
  bulk_load(st->u, a.in.u + off, bytes, bar);
  bulk_load(st->v, a.in.v + off, bytes, bar);
  bulk_load(st->w, a.in.w + off, bytes, bar);
  if (a.in.id) bulk_load(st->id, a.in.id + off, bytes, bar);
}

template <int B, int I>
__device__ __forceinline__ void read_striped_smem(const uint32_t *p, uint32_t (&x)[I]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
  for (int c = 0; c < I / 4; ++c) {
    const uint4 t = q[c * B + threadIdx.x];
    x[4 * c] = t.x;
    x[4 * c + 1] = t.y;
    x[4 * c + 2] = t.z;
    x[4 * c + 3] = t.w;
  }
}

// Input stages plus one output stage of T items.  (Two input stages for the
// partition, at two blocks per SM, measured slower on GB300: 1.35 against
// 1.04 ms per C3 solve.)
template <int B, int I>
constexpr size_t tma_smem_bytes() { return sizeof(EdgeStage<B * I>) * (TMA_STAGES + 1); }

template <int MODE, int B, int I>
__global__ void __launch_bounds__(B, Shape<B, I>::minb(Shape<B, I>::tma_regs)) compact_tma_kernel(CompactArgs a) {
  constexpr int T = Shape<B, I>::T;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  EdgeStage<T> *stage = reinterpret_cast<EdgeStage<T> *>(smem_dyn);  // TMA_STAGES input stages + 1 output stage
  EdgeStage<T> *out = stage + TMA_STAGES;
  __shared__ __align__(8) u64 mbar[TMA_STAGES];
  __shared__ uint32_t s_warp[B / 32 + 1];
  __shared__ uint32_t s_base[1];
  __shared__ uint32_t s_abort;

  const uint64_t m = a.m_dev ? min((uint64_t)*a.m_dev, a.m) : a.m;
  const uint64_t ntiles = (m + T - 1) / T, nfull = m / T;
  const uint64_t G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TMA_STAGES; ++s) mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    for (int s = 0; s < TMA_STAGES; ++s) {
      const uint64_t tile = blockIdx.x + (uint64_t)s * G;
      if (tile < nfull) issue_tile<T>(a, tile, &stage[s], &mbar[s]);
    }
  }
  __syncthreads();
  const u64 pivot = compact_pivot(a, MODE);
  uint64_t it = 0;
  for (;; ++it) {
    const uint64_t tile = blockIdx.x + it * G;
    if (tile >= ntiles) break;
    const int si = (int)(it % TMA_STAGES);
    EdgeStage<T> *st = &stage[si];
    const uint64_t tb = tile * T;
    uint32_t eu[I], ev[I], ew[I], ei[I];
    if (tile < nfull) {
      if (!mbar_wait_bounded(&mbar[si], (uint32_t)((it / TMA_STAGES) & 1))) atomicOr(&s_abort, 1u);
      __syncthreads();
      if (s_abort) break;
      read_striped_smem<B, I>(st->u, eu);
      read_striped_smem<B, I>(st->v, ev);
      read_striped_smem<B, I>(st->w, ew);
      if (a.in.id) {
        read_striped_smem<B, I>(st->id, ei);
      } else {
#pragma unroll
        for (int k = 0; k < I; ++k) ei[k] = (uint32_t)(tb + item_off<B>(k));
      }
      __syncthreads();  // the stage is consumed: refill it with the tile TMA_STAGES ahead
      if (threadIdx.x == 0) {
        const uint64_t next = tile + (uint64_t)TMA_STAGES * G;
        if (next < nfull) issue_tile<T>(a, next, st, &mbar[si]);
      }
    } else {  // the partial last tile: plain loads
#pragma unroll
      for (int k = 0; k < I; ++k) {
        const uint64_t j = tb + item_off<B>(k);
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
    const uint32_t valid = valid_items_s<B, I>(tb, m);
    const uint32_t keep = keep_flags<MODE>(a, valid, pivot, eu, ev, ew, ei, a.giant_bits);
    if (a.max_w) {
      uint32_t mx = 0;
#pragma unroll
      for (int k = 0; k < I; ++k) mx = max(mx, (valid >> k & 1) ? ew[k] : 0u);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0 && mx > __ldca(a.max_w)) atomicMax(a.max_w, mx);
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan<B>((uint32_t)__popc(keep), total, s_warp);
    const uint64_t obase = tile_claim(a.st.total, total, s_base);
    emit_survivors<B, I>(a, keep, excl, within_capacity(a, obase, total), obase, eu, ev, ew, ei, out->u, out->v,
                         out->w, out->id);
    __syncthreads();  // the output stage is reused by the next tile
  }
  // On an abort the block's remaining tiles were not compacted: latch the
  // error (the solve then fails instead of returning a short list), and wait
  // (bounded) for the copies this block still has in flight before its shared
  // memory goes away.
  __syncthreads();
  if (s_abort && threadIdx.x == 0) {
    atomicOr(a.st.err, ERR_TMA);
    for (uint64_t k = it; k < it + TMA_STAGES; ++k) {
      const uint64_t tile = blockIdx.x + k * G;
      if (tile < nfull) mbar_wait_bounded(&mbar[k % TMA_STAGES], (uint32_t)((k / TMA_STAGES) & 1));
    }
  }
}

// ------------------------------------------------- warp-streamed passes

// The filter keeps few of the edges it reads (on RMAT about 2% of a level's
// list: the heavy edges between different components of the light forest,
// Thm. 1), so its pass is a stream with gathers more than a compaction, and
// the gathers (giant-component bitmap words, then labels) set its speed.  Here
// every warp streams its own tiles of 32 x I edges: warp gw of the G warps in
// the grid takes tiles gw, gw + G, gw + 2G, ...; a full tile arrives in one of
// the warp's S shared-memory stages by bulk copies (one per array, completion
// counted on the stage's mbarrier) issued S tiles ahead, and the stage is
// refilled as soon as the tile is in registers, so the next tile's copy
// overlaps this tile's gathers.  The warp's survivors go to its own O-entry
// staging buffer, which is written out (one atomic claim of output slots,
// coalesced stores, then the best[] relaxation and recorded ends) when it
// fills and when the warp finishes.  No block-wide barrier is on the path: a
// warp waiting on its gathers never holds up another.
//
// The filter's shape is measured on GB300 (RMAT n=2^24, m=2^28, median pivots, filter class
// per solve): 32 warps x 4 edges per lane, one stage: 2.49 ms; 16 warps x 8,
// two blocks per SM: 2.49; 24 x 8, one stage: 2.58; 24 x 8, two stages: 4.39;
// the block-synchronous compaction kernel: 4.02.  Shared memory is the lever:
// the rest of the SM's 256 KB is L1, which serves the hub vertices' bitmap
// words and labels, so a deep ring (216 KB) lost to a single stage (80 KB).
template <int W, int I, int S, int O, int MINB>
struct WarpShape {
  static constexpr int warps = W, items = I, stages = S, out = O, minb = MINB;
  static constexpr int threads = W * 32;
  static constexpr int tile = 32 * I;  // edges per warp tile
  struct __align__(16) Stage {
    uint32_t u[tile], v[tile], w[tile], id[tile];
  };
  struct __align__(16) Out {
    uint32_t u[O], v[O], w[O], id[O];
  };
  static constexpr size_t smem = sizeof(Stage) * S * W + sizeof(Out) * W;
};
// Its staging buffer holds 64 survivors per warp: every flush claims output
// slots with one atomic add on the list counter, and with 1/8-quantile pivots
// (the top level filters 7/8 of the input) 32 per warp made those adds queue
// (filter class 2.49 ms; 64: 2.37; 96: 2.39; 128: 2.42, less L1).
using FilterWarp = WarpShape<32, 4, 1, 64, 1>;
// The partition keeps the light share q of its list (1/8 by default), so it
// streams with sparse survivors too.  Its survivors are denser than the
// filter's, and every flush claims its output slots with one atomic add on the
// list counter, so its staging buffer is large.  Measured on GB300 (RMAT
// n=2^24, m=2^28, partition class per solve): 24 warps x 8 edges per lane with
// 32 / 64 / 128 / 192 / 256 staged survivors per warp: 2.23 / 0.89 / 0.79 /
// 0.78 / 0.87 ms (256 leaves little L1); 32 x 4 with 64: 0.98, two stages:
// 0.97; 16 x 8 with 256: 0.86; the block kernel (256 x 8): 1.04.  At larger
// light shares the claims pile up (batched mix: 2.69 ms at q = 1/4, 6.24 ms at
// q = 1/2), so the solver uses this pass only for q up to 1/8.
using PartitionWarp = WarpShape<24, 8, 1, 128, 1>;

// Item k of lane l in a warp tile sits at (k / 4) * 128 + 4 l + k % 4, so each
// 16-byte shared-memory read of the warp covers 512 contiguous bytes.
__device__ __forceinline__ uint32_t witem_off(int k) {
  return (uint32_t)((k >> 2) * 128 + 4 * (threadIdx.x & 31) + (k & 3));
}

template <int I>
__device__ __forceinline__ void read_wstage(const uint32_t *p, uint32_t (&x)[I]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < I / 4; ++c) {
    const uint4 t = q[32 * c + lane];
    x[4 * c] = t.x;
    x[4 * c + 1] = t.y;
    x[4 * c + 2] = t.z;
    x[4 * c + 3] = t.w;
  }
}

// Issues the bulk copies of full warp tile `tile` into stage `st` (one lane).
template <class WS>
__device__ __forceinline__ void issue_wtile(const CompactArgs &a, uint64_t tile, typename WS::Stage *st, u64 *bar) {
  const uint32_t bytes = WS::tile * 4;
  const uint64_t off = tile * WS::tile;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order the stage's earlier generic reads
  mbar_arrive_expect_tx(bar, (a.in.id ? 4u : 3u) * bytes);
  bulk_load(st->u, a.in.u + off, bytes, bar);
  bulk_load(st->v, a.in.v + off, bytes, bar);
  bulk_load(st->w, a.in.w + off, bytes, bar);
  if (a.in.id) bulk_load(st->id, a.in.id + off, bytes, bar);
}

// Writes the warp's `count` staged survivors to the output list (all lanes).
template <class WS>
__device__ __forceinline__ void warp_flush(const CompactArgs &a, const typename WS::Out *o, uint32_t count) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(a.st.total, (unsigned long long)count);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (a.out_cap && base + count > a.out_cap) {  // past the output capacity: write the part that fits
    if (lane == 0) atomicOr(a.st.err, ERR_OVERFLOW);
    count = base < a.out_cap ? (uint32_t)(a.out_cap - base) : 0u;
  }
  for (uint32_t i = lane; i < count; i += 32) {
    const uint32_t x = o->u[i], y = o->v[i], w = o->w[i], id = o->id[i];
    a.out.u[base + i] = x;
    a.out.v[base + i] = y;
    a.out.w[base + i] = w;
    a.out.id[base + i] = id;
    if (a.cur_u) {  // ends by id, for the hook of the round that relaxes this list
      a.cur_u[id] = x;
      a.cur_v[id] = y;
    }
    if (a.best) {  // the next round's minEdges, fused
      const u64 kx = relax_key(a.kl, w, id, y), ky = relax_key(a.kl, w, id, x);
      const u64 cx = __ldca(a.best + x), cy = __ldca(a.best + y);
      if (kx < cx) atomicMin(a.best + x, kx);
      if (ky < cy) atomicMin(a.best + y, ky);
    }
  }
  __syncwarp();  // the staging buffer is refilled next
}

template <int MODE, class WS>
__global__ void __launch_bounds__(WS::threads, WS::minb) stream_warp_kernel(CompactArgs a) {
  static_assert(MODE == CM_FILTER || MODE == CM_HEAVY || MODE == CM_PARTITION,
                "the warp-streamed pass serves the filter modes and the partition");
  constexpr int I = WS::items, S = WS::stages, O = WS::out, T = WS::tile;
  using Stage = typename WS::Stage;
  using Out = typename WS::Out;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  __shared__ __align__(8) u64 mbar[WS::warps][S];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Stage *stage = reinterpret_cast<Stage *>(smem_dyn) + wid * S;
  Out *o = reinterpret_cast<Out *>(smem_dyn + sizeof(Stage) * S * WS::warps) + wid;
  u64 *bar = mbar[wid];

  const uint64_t m = a.m_dev ? min((uint64_t)*a.m_dev, a.m) : a.m;
  const uint64_t ntiles = (m + T - 1) / T, nfull = m / T;
  const uint64_t G = (uint64_t)gridDim.x * WS::warps;
  const uint64_t gw = (uint64_t)blockIdx.x * WS::warps + wid;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < S; ++s) {
      const uint64_t tile = gw + (uint64_t)s * G;
      if (tile < nfull) issue_wtile<WS>(a, tile, &stage[s], &bar[s]);
    }
  }
  __syncwarp();
  const u64 pivot = compact_pivot(a, MODE);
  // the giant-component bitmap, unless too few sampled edge ends lie in that
  // component for its test to spare label gathers
  const uint32_t *gbits = (a.giant_count && __ldg(a.giant_count) < GIANT_MIN_COUNT) ? nullptr : a.giant_bits;
  uint32_t fill = 0;  // staged survivors (the same in every lane)
  uint32_t wmax = 0;  // largest weight this lane read (partition with a.max_w)
  bool abort = false;
  uint64_t it = 0;
  for (;; ++it) {
    const uint64_t tile = gw + it * G;
    if (tile >= ntiles) break;
    const uint64_t tb = tile * T;
    uint32_t eu[I], ev[I], ew[I], ei[I];
    uint32_t valid = (I >= 32 ? 0xffffffffu : (1u << I) - 1u);
    if (tile < nfull) {
      const int si = (int)(it % S);
      Stage *st = &stage[si];
      const bool ok = mbar_wait_bounded(&bar[si], (uint32_t)((it / S) & 1));
      if (!__all_sync(0xffffffffu, ok)) {
        abort = true;
        break;
      }
      read_wstage<I>(st->u, eu);
      read_wstage<I>(st->v, ev);
      read_wstage<I>(st->w, ew);
      if (a.in.id) {
        read_wstage<I>(st->id, ei);
      } else {
#pragma unroll
        for (int k = 0; k < I; ++k) ei[k] = (uint32_t)(tb + witem_off(k));
      }
      __syncwarp();  // every lane has the tile: refill the stage with the tile S ahead
      if (lane == 0) {
        const uint64_t next = tile + (uint64_t)S * G;
        if (next < nfull) issue_wtile<WS>(a, next, st, &bar[si]);
      }
    } else {  // the partial last tile: plain loads
      valid = 0;
#pragma unroll
      for (int k = 0; k < I; ++k) {
        const uint64_t j = tb + witem_off(k);
        if (j < m) {
          eu[k] = __ldg(a.in.u + j);
          ev[k] = __ldg(a.in.v + j);
          ew[k] = __ldg(a.in.w + j);
          ei[k] = a.in.id ? __ldg(a.in.id + j) : (uint32_t)j;
          valid |= 1u << k;
        } else {
          eu[k] = ev[k] = ew[k] = ei[k] = 0;
        }
      }
    }
    const uint32_t keep = keep_flags<MODE>(a, valid, pivot, eu, ev, ew, ei, gbits);
    if (MODE == CM_PARTITION && a.max_w) {
#pragma unroll
      for (int k = 0; k < I; ++k) wmax = max(wmax, (valid >> k & 1) ? ew[k] : 0u);
    }
    // warp-wide exclusive prefix of the kept counts: survivor ranks 0..total-1
    const uint32_t c = (uint32_t)__popc(keep);
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31), excl = incl - c;
    // append the ranks [lo, lo + take) to the free part of the staging buffer
    for (uint32_t lo = 0; lo < total;) {
      const uint32_t take = min((uint32_t)O - fill, total - lo);
#pragma unroll
      for (int k = 0; k < I; ++k) {
        if (!(keep >> k & 1)) continue;
        const uint32_t r = excl + (uint32_t)__popc(keep & ((1u << k) - 1u));
        if (r >= lo && r < lo + take) {
          const uint32_t p = fill + r - lo;
          o->u[p] = eu[k];
          o->v[p] = ev[k];
          o->w[p] = ew[k];
          o->id[p] = ei[k];
        }
      }
      __syncwarp();
      fill += take;
      lo += take;
      if (fill == (uint32_t)O) {
        warp_flush<WS>(a, o, fill);
        fill = 0;
      }
    }
  }
  if (!abort) {
    if (fill) warp_flush<WS>(a, o, fill);
    if (MODE == CM_PARTITION && a.max_w) {  // the input's largest weight (key layout), one atomic per warp
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, d));
      if (lane == 0 && wmax > __ldca(a.max_w)) atomicMax(a.max_w, wmax);
    }
    return;
  }
  // A bulk copy never completed: this warp's remaining tiles were not read.
  // Latch the error (the solve fails instead of returning a short list) and
  // wait (bounded) for the copies still in flight into this warp's stages
  // before the block's shared memory goes away.
  if (lane == 0) {
    atomicOr(a.st.err, ERR_TMA);
    for (uint64_t k = it; k < it + S; ++k) {
      const uint64_t tile = gw + k * G;
      if (tile < nfull) mbar_wait_bounded(&bar[k % S], (uint32_t)((k / S) & 1));
    }
  }
  __syncwarp();
}

// --------------------------------------------------------------- min edges

// minEdges of a round that starts from a stored list (the input, or a list
// built by partition/filter): best[c] = min slot key over incident edges.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK) min_edges_kernel(EdgeList in, uint64_t m, uint32_t n, int validate,
                                                          KeyLayout kl, u64 *best, uint32_t *err) {
  const uint64_t ntiles = (m + TILE - 1) / TILE;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t tb = tile * TILE;
    uint32_t eu[ITEMS], ev[ITEMS], ew[ITEMS], ei[ITEMS];
    if (VEC && tb + TILE <= m) {
      load_striped(in.u, tb, eu);
      load_striped(in.v, tb, ev);
      load_striped(in.w, tb, ew);
      if (in.id) load_striped(in.id, tb, ei);
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const uint64_t j = tb + item_off(k);
        eu[k] = j < m ? __ldg(in.u + j) : 0u;
        ev[k] = j < m ? __ldg(in.v + j) : 0u;
        ew[k] = j < m ? __ldg(in.w + j) : 0u;
        if (in.id) ei[k] = j < m ? __ldg(in.id + j) : 0u;
      }
    }
    if (!in.id) {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) ei[k] = (uint32_t)(tb + item_off(k));
    }
    uint32_t mask = 0;
    u64 key[ITEMS], keyb[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint64_t j = tb + item_off(k);
      bool ok = j < m;
      if (ok && validate && (eu[k] >= n || ev[k] >= n)) {
        atomicOr(err, ERR_VERTEX);
        ok = false;
      }
      ok = ok && eu[k] != ev[k];
      mask |= (ok ? 1u : 0u) << k;
      key[k] = relax_key(kl, ew[k], ei[k], ev[k]);
      keyb[k] = relax_key(kl, ew[k], ei[k], eu[k]);
    }
    relax_pairs(best, eu, ev, key, keyb, mask);
  }
}

// Adds this thread's sum of chosen weights into a spread counter: one atomic
// per warp (all 32 lanes call together).
__device__ __forceinline__ void wsum_add(u64 *wsum, u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (wsum && (threadIdx.x & 31) == 0 && v)
    atomicAdd(reinterpret_cast<unsigned long long *>(wsum) +
                  ((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (WSUM_SLOTS - 1)),
              (unsigned long long)v);
}

// -------------------------------------------------------------------- hook

constexpr uint32_t FIND_STEPS = 1u << 12;  // bound on one parent-chain walk

// Hooking (Section 2.3 / 4.2) over the candidate vertices: a vertex c with
// best[c] != INF points to the other end of its minimum edge e; in a 2-cycle
// (both ends chose the same edge) the smaller vertex stays root.  Each chosen
// edge's id is set once in the bitmap (by the vertex that is not the root).
// The active vertices (best != INF) are compacted into active_out.
//
// IOTA: the candidates are 0..ncand-1 (a call's first round), else the list
// cand.  PACKED: the key holds the other end (see KeyLayout), so no walk is
// needed and this instantiation keeps few registers (6 blocks per SM).
//
// Otherwise the ends of e are found through the ends recorded by id (or the
// input arrays): src[e] and dst[e] are vertices whose current labels are
// reached by following parent pointers until the first vertex that is active
// this round (best != INF).
// Every vertex passed on the way was merged in an earlier round and has no edge
// now, and best[] is not written during the hook, so the hooks of other threads
// (which only change parent[] of active vertices) cannot redirect a walk.  All
// 2 * ITEMS walks of a thread advance in lockstep, so each step costs one round
// of independent loads.  The start vertex of a walk longer than one step is
// then pointed at its label directly (a concurrent walker sees either pointer,
// both on the same path).
template <bool IOTA, bool PACKED, int B, int I>
__global__ void __launch_bounds__(B, Shape<B, I>::minb(PACKED ? Shape<B, I>::hook_packed_regs
                                                                  : Shape<B, I>::hook_regs)) hook_kernel(HookArgs a) {
  constexpr int T = Shape<B, I>::T;
  __shared__ uint32_t s_c[T];
  __shared__ uint32_t s_warp[B / 32 + 1];
  __shared__ uint32_t s_base[1];

  const uint64_t nc = a.ncand_dev ? *a.ncand_dev : a.ncand;
  const int wshift = PACKED ? a.kl.idbits + a.kl.vbits : 32;  // the weight's place in a key
  u64 wacc = 0;  // weights of the edges this thread chose
  for (uint64_t tile = blockIdx.x; tile * T < nc; tile += gridDim.x) {  // uniform per block
  const uint64_t tb = tile * T;
  uint32_t c[I];
  u64 kk[I];
  if (!IOTA && tb + T <= nc && (((uintptr_t)a.cand) & 15u) == 0) {
    load_striped<B, I>(a.cand, tb, c);
  } else {
#pragma unroll
    for (int k = 0; k < I; ++k) {
      const uint64_t j = tb + item_off<B>(k);
      c[k] = IOTA ? (uint32_t)j : (j < nc ? __ldg(a.cand + j) : 0u);
    }
  }
#pragma unroll
  for (int k = 0; k < I; ++k) kk[k] = (tb + item_off<B>(k) < nc) ? a.best[c[k]] : KEY_INF;
  uint32_t keep = 0;
  if (PACKED) {  // the chosen neighbour is in the key (a.kl.packed)
#pragma unroll
    for (int k = 0; k < I; ++k) {
      if (kk[k] == KEY_INF) continue;
      keep |= 1u << k;
      const uint32_t e = key_edge_id(a.kl, kk[k]);
      const uint32_t other = (uint32_t)(kk[k] & ((1ULL << a.kl.vbits) - 1));
      const bool root = same_edge(a.kl, a.best[other], kk[k]) && c[k] < other;
      a.parent[c[k]] = root ? c[k] : other;
      if (!root) {
        atomicOr(a.chosen_bits + (e >> 5), 1u << (e & 31));
        wacc += kk[k] >> wshift;
      }
    }
  } else {
  uint32_t start[2 * I], cur[2 * I];
#pragma unroll
  for (int k = 0; k < I; ++k) {
    keep |= (kk[k] != KEY_INF ? 1u : 0u) << k;
    const uint32_t e = (uint32_t)kk[k];
    start[2 * k] = kk[k] != KEY_INF ? __ldg(a.src + e) : c[k];
    start[2 * k + 1] = kk[k] != KEY_INF ? __ldg(a.dst + e) : c[k];
  }
  // lockstep walks to the current labels
  uint32_t pending = 0;
#pragma unroll
  for (int i = 0; i < 2 * I; ++i) {
    cur[i] = start[i];
    pending |= ((keep >> (i >> 1)) & 1u) << i;
  }
  uint32_t steps = 0;
  while (pending) {
    if (++steps > FIND_STEPS) {
      atomicOr(a.err, ERR_JUMP);
      break;
    }
    u64 bv[2 * I];
    uint32_t pv[2 * I];
#pragma unroll
    for (int i = 0; i < 2 * I; ++i) {
      bv[i] = (pending >> i & 1) ? a.best[cur[i]] : 0ULL;
      pv[i] = (pending >> i & 1) ? __ldcg(a.parent + cur[i]) : 0u;
    }
#pragma unroll
    for (int i = 0; i < 2 * I; ++i) {
      if (!(pending >> i & 1)) continue;
      if (bv[i] != KEY_INF || pv[i] == cur[i])
        pending &= ~(1u << i);
      else
        cur[i] = pv[i];
    }
  }
#pragma unroll
  for (int k = 0; k < I; ++k) {
    if (!(keep >> k & 1)) continue;
    const uint32_t e = (uint32_t)kk[k];
    const uint32_t other = cur[2 * k] ^ cur[2 * k + 1] ^ c[k];
    const bool root = a.best[other] == kk[k] && c[k] < other;
    a.parent[c[k]] = root ? c[k] : other;
    if (!root) {
      atomicOr(a.chosen_bits + (e >> 5), 1u << (e & 31));
      wacc += kk[k] >> wshift;
    }
  }
  // shortcut the walked start vertices to their labels
#pragma unroll
  for (int i = 0; i < 2 * I; ++i)
    if ((keep >> (i >> 1) & 1) && cur[i] != start[i] && __ldcg(a.parent + start[i]) != cur[i])
      __stcg(a.parent + start[i], cur[i]);
  }

  uint32_t total;
  const uint32_t excl = block_exclusive_scan<B>((uint32_t)__popc(keep), total, s_warp);
  const uint64_t obase = tile_claim(a.counter, total, s_base);
#pragma unroll
  for (int k = 0; k < I; ++k)
    if (keep >> k & 1) s_c[excl + (uint32_t)__popc(keep & ((1u << k) - 1u))] = c[k];
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < total; i += B) a.active_out[obase + i] = s_c[i];
  __syncthreads();  // s_c, s_warp and s_base are reused by the block's next tile
  }
  wsum_add(a.wsum, wacc);
}

// --------------------------------------------------------- pointer jumping

// Pointer doubling toward the roots (Section 4.2): each listed vertex follows
// parent pointers (reading the other threads' progress) for at most max_steps
// steps and stores the furthest ancestor reached; `flag` is set if some vertex
// did not reach its root, and the host launches again.  Parent values only ever
// move toward the root and no root changes during a jump, so concurrent reads
// and writes are benign, and so is a stale copy: the step loads go through L1,
// which keeps the many reads of a large component's root (every walk in that
// component ends there) off a single L2 slice.  When
// reset_best is set, best[c] is returned to INF for the next round.
constexpr int JUMP_ITEMS = 4;                   // vertices per thread, walked in lockstep
constexpr int JUMP_TILE = BLOCK * JUMP_ITEMS;

__global__ void __launch_bounds__(BLOCK) jump_kernel(const uint32_t *act, const u64 *count_dev, uint64_t count_host,
                                                     uint32_t *parent, u64 *best, int reset_best, uint32_t *flag,
                                                     uint32_t max_steps) {
  const uint64_t cnt = count_dev ? *count_dev : count_host;
  // each thread takes JUMP_ITEMS vertices of a block tile (striped, so the list
  // and parent[] reads are coalesced) and advances their walks together: every
  // step issues up to JUMP_ITEMS independent loads instead of one
  for (uint64_t tb = (uint64_t)blockIdx.x * JUMP_TILE; tb < cnt; tb += (uint64_t)gridDim.x * JUMP_TILE) {
    uint32_t c[JUMP_ITEMS], p[JUMP_ITEMS];
    uint32_t live = 0;
#pragma unroll
    for (int k = 0; k < JUMP_ITEMS; ++k) {
      const uint64_t i = tb + (uint64_t)k * BLOCK + threadIdx.x;
      const bool ok = i < cnt;
      c[k] = ok ? (act ? __ldg(act + i) : (uint32_t)i) : 0u;
      live |= (ok ? 1u : 0u) << k;
    }
#pragma unroll
    for (int k = 0; k < JUMP_ITEMS; ++k) {
      p[k] = (live >> k & 1) ? __ldcg(parent + c[k]) : 0u;
      if (reset_best && (live >> k & 1)) best[c[k]] = KEY_INF;
    }
    uint32_t pending = live, moved = 0;
    for (uint32_t steps = 0; pending && steps < max_steps; ++steps) {
      uint32_t pp[JUMP_ITEMS];
#pragma unroll
      for (int k = 0; k < JUMP_ITEMS; ++k) pp[k] = (pending >> k & 1) ? __ldca(parent + p[k]) : 0u;
#pragma unroll
      for (int k = 0; k < JUMP_ITEMS; ++k) {
        if (!(pending >> k & 1)) continue;
        if (pp[k] == p[k]) {
          pending &= ~(1u << k);
        } else {
          p[k] = pp[k];
          moved |= 1u << k;
        }
      }
    }
    if (pending) atomicOr(flag, 1u);
#pragma unroll
    for (int k = 0; k < JUMP_ITEMS; ++k)
      if (moved >> k & 1) __stcg(parent + c[k], p[k]);
  }
}

// The same over all n vertices (no list): lane l of a warp takes the four
// consecutive vertices 4q..4q+3 (one 16-byte load and, if one moved, one
// 16-byte store of parent), so that the pass is a plain stream plus the walk
// steps, which mostly hit L1 (most walks end at a few large components'
// roots).  Warps stride over warp-aligned bases and stay converged; with
// gbits, eight lanes' four marks form one 32-vertex bitmap word.
__global__ void __launch_bounds__(BLOCK) jump_all_kernel(uint32_t *parent, u64 *best, int reset_best, uint64_t n,
                                                         uint32_t *flag, uint32_t max_steps, const uint32_t *groot,
                                                         uint32_t *gbits) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nq = (n + 3) / 4;
  const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
  const bool vec = aligned16_dev(parent);
  const uint32_t r = gbits ? *groot : 0u;
  for (uint64_t qb = (uint64_t)blockIdx.x * BLOCK + (threadIdx.x & ~31u); qb < nq; qb += stride) {  // uniform per warp
    const uint64_t q = qb + lane, c0 = 4 * q;
    const bool full = vec && c0 + 4 <= n;
    uint32_t p[4];
    uint32_t live = 0;
    if (full) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(parent) + q);
      p[0] = v.x; p[1] = v.y; p[2] = v.z; p[3] = v.w;
      live = 0xfu;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = c0 + k < n;
        p[k] = ok ? __ldcg(parent + c0 + k) : 0u;
        live |= (ok ? 1u : 0u) << k;
      }
    }
    if (reset_best) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (live >> k & 1) best[c0 + k] = KEY_INF;
    }
    uint32_t pending = live, moved = 0;
    for (uint32_t steps = 0; pending && steps < max_steps; ++steps) {
      uint32_t pp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) pp[k] = (pending >> k & 1) ? __ldca(parent + p[k]) : 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!(pending >> k & 1)) continue;
        if (pp[k] == p[k]) {
          pending &= ~(1u << k);
        } else {
          p[k] = pp[k];
          moved |= 1u << k;
        }
      }
    }
    if (pending) atomicOr(flag, 1u);
    if (moved) {
      if (full) {
        __stcg(reinterpret_cast<uint4 *>(parent) + q, make_uint4(p[0], p[1], p[2], p[3]));
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (moved >> k & 1) __stcg(parent + c0 + k, p[k]);
      }
    }
    if (gbits) {
      uint32_t nib = 0;  // an unfinished walk marks nothing
#pragma unroll
      for (int k = 0; k < 4; ++k) nib |= (((live & ~pending) >> k & 1) && p[k] == r ? 1u : 0u) << k;
      uint32_t word = nib << (4 * (lane & 7u));
      word |= __shfl_xor_sync(0xffffffffu, word, 1);
      word |= __shfl_xor_sync(0xffffffffu, word, 2);
      word |= __shfl_xor_sync(0xffffffffu, word, 4);
      const uint64_t wi = (qb >> 3) + (lane >> 3);  // vertices 32 wi .. 32 wi + 31
      if ((lane & 7u) == 0 && 32 * wi < n) gbits[wi] = word;
    }
  }
}

// ------------------------------------------------------------- small kernels

__global__ void hash_insert_kernel(EdgeList in, uint64_t m, HashSlot *table, uint64_t tmask, uint32_t *err) {
  for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < m; j += (uint64_t)gridDim.x * BLOCK) {
    const uint32_t u = in.u[j], v = in.v[j];
    if (u == v) continue;
    if (!hash_insert(table, tmask, pair_of(u, v), edge_key(in.w[j], in.id ? in.id[j] : (uint32_t)j)))
      atomicOr(err, ERR_HASH);
  }
}

__global__ void __launch_bounds__(BLOCK) max_weight_kernel(const uint32_t *w, uint64_t m, uint32_t *out) {
  uint32_t mx = 0;
  const uint64_t nv = ((uintptr_t)w & 15u) ? 0 : m / 4;  // 16-byte vectors
  const uint4 *w4 = reinterpret_cast<const uint4 *>(w);
  const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
  uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  for (; i + 3 * stride < nv; i += 4 * stride) {
    const uint4 a = __ldcs(w4 + i), b = __ldcs(w4 + i + stride), c = __ldcs(w4 + i + 2 * stride),
                d = __ldcs(w4 + i + 3 * stride);
    mx = max(mx, max(max(max(a.x, a.y), max(a.z, a.w)), max(max(b.x, b.y), max(b.z, b.w))));
    mx = max(mx, max(max(max(c.x, c.y), max(c.z, c.w)), max(max(d.x, d.y), max(d.z, d.w))));
  }
  for (; i < nv; i += stride) {
    const uint4 a = __ldcs(w4 + i);
    mx = max(mx, max(max(a.x, a.y), max(a.z, a.w)));
  }
  for (uint64_t j = nv * 4 + (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < m; j += stride) mx = max(mx, w[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// Sets ERR_VERTEX if some x[i] (i < count) is >= bound.
__global__ void range_check_kernel(const uint32_t *x, uint64_t count, uint32_t bound, uint32_t *err) {
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < count; i += (uint64_t)gridDim.x * BLOCK)
    bad |= __ldcs(x + i) >= bound;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_VERTEX);
}

__global__ void iota_kernel(uint32_t *p, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (uint64_t)gridDim.x * BLOCK)
    p[i] = (uint32_t)i;
}


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

// The sample key of rank `rank` (0-based, < sample; sample / 2 is the median
// of Alg. 2), by radix selection in one block: bytes are fixed from the most
// significant one that differs between the sample's minimum and maximum,
// using a 256-bin histogram per byte.
constexpr int SEL_THREADS = 1024;
__global__ void __launch_bounds__(SEL_THREADS) pivot_select_kernel(const u64 *keys, uint32_t sample, uint32_t rank0,
                                                                   u64 *out) {
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
    s_rank = rank0;
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

// The same selection spread over PSEL_BLOCKS blocks of a cooperative launch:
// every thread draws its samples, then each pass histograms the next 12 bits
// (below the bits shared by all candidates) in shared memory, adds the block's
// bins to a global histogram, and after a grid-wide barrier every block reads
// the histogram and fixes the same digit.  The first pass starts below the
// bits that the sample's minimum and maximum share.
constexpr int PSEL_BLOCKS = 64, PSEL_THREADS = 1024, PSEL_BITS = 12, PSEL_BINS = 1 << PSEL_BITS;

struct PivotScratch {
  u64 min, max;
  uint32_t hist[2][PSEL_BINS];
};

__global__ void __launch_bounds__(PSEL_THREADS) pivot_coop_kernel(EdgeList in, uint64_t m_bound, const u64 *m_dev,
                                                                 u64 state, uint32_t sample, uint32_t rank0,
                                                                 u64 *keys, PivotScratch *ps, u64 *out) {
  const uint64_t m = m_dev ? min((uint64_t)*m_dev, m_bound) : m_bound;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ uint32_t s_hist[PSEL_BINS];
  __shared__ u64 s_prefix, s_mask;
  __shared__ uint32_t s_rank, s_scan[PSEL_THREADS / 32 + 1];
  const uint32_t nthreads = PSEL_BLOCKS * PSEL_THREADS;
  const uint32_t tid = blockIdx.x * PSEL_THREADS + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < 2 * PSEL_BINS; i += PSEL_THREADS) (&ps->hist[0][0])[i] = 0;
    if (threadIdx.x == 0) {
      ps->min = KEY_INF;
      ps->max = 0;
    }
  }
  grid.sync();
  // draw the samples; track the minimum and maximum key
  u64 mn = KEY_INF, mx = 0;
  for (uint32_t i = tid; i < sample; i += nthreads) {
    u64 k = KEY_INF;
    if (m) {
      const uint64_t j = __umul64hi(splitmix64_at(state, i), m);
      k = ((u64)__ldg(in.w + j) << 32) | (u64)(in.id ? __ldg(in.id + j) : (uint32_t)j);
    }
    keys[i] = k;
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
    atomicMin(&ps->min, mn);
    atomicMax(&ps->max, mx);
  }
  grid.sync();
  mn = *(volatile u64 *)&ps->min;
  mx = *(volatile u64 *)&ps->max;
  if (mn == mx || sample == 0) {
    if (tid == 0) *out = mn;
    return;
  }
  int low = 63 - __clzll((long long)(mn ^ mx)) + 1 - PSEL_BITS;  // lowest bit of the first digit
  if (threadIdx.x == 0) {
    const int top = low + PSEL_BITS;  // bits >= top are shared by every key
    s_mask = top >= 64 ? 0ULL : ~((1ULL << top) - 1ULL);
    s_prefix = mn & s_mask;
    s_rank = rank0;
  }
  __syncthreads();
  for (int pass = 0;; ++pass) {
    const int shift = low < 0 ? 0 : low;
    const int width = low < 0 ? PSEL_BITS + low : PSEL_BITS;
    const uint32_t dmask = (1u << width) - 1u;
    for (int i = threadIdx.x; i < PSEL_BINS; i += PSEL_THREADS) s_hist[i] = 0;
    __syncthreads();
    const u64 prefix = s_prefix, mask = s_mask;
    for (uint32_t i = tid; i < sample; i += nthreads) {
      const u64 k = keys[i];
      if ((k & mask) == prefix) atomicAdd(&s_hist[(uint32_t)(k >> shift) & dmask], 1u);
    }
    __syncthreads();
    uint32_t *gh = ps->hist[pass & 1];
    for (int i = threadIdx.x; i < PSEL_BINS; i += PSEL_THREADS)
      if (s_hist[i]) atomicAdd(gh + i, s_hist[i]);
    grid.sync();
    // every block: find the digit holding the current rank (4 bins per thread)
    uint32_t c4[4], sum = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      c4[b] = *(volatile uint32_t *)(gh + threadIdx.x * 4 + b);
      sum += c4[b];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_scan[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const uint32_t v = lane < PSEL_THREADS / 32 ? s_scan[lane] : 0u;
      uint32_t wi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < PSEL_THREADS / 32) s_scan[lane] = wi - v;
    }
    __syncthreads();
    const uint32_t before = s_scan[wid] + incl - sum, rank = s_rank;
    if (before <= rank && rank < before + sum) {  // exactly one thread
      uint32_t below = before;
      int b = 0;
      while (below + c4[b] <= rank) below += c4[b++];
      s_prefix = prefix | ((u64)(threadIdx.x * 4 + b) << shift);
      s_mask = mask | ((u64)dmask << shift);
      s_rank = rank - below;
    }
    if (blockIdx.x == 0)  // the other histogram is reused by the next pass
      for (int i = threadIdx.x; i < PSEL_BINS; i += PSEL_THREADS) ps->hist[(pass + 1) & 1][i] = 0;
    __syncthreads();
    if (shift == 0) break;
    low -= PSEL_BITS;
    grid.sync();
  }
  if (tid == 0) *out = s_prefix;
}

// ---------------------------------------------------- tile-local contraction

// Local preprocessing (Section 4.1) with vertex-range tiles standing in for the
// paper's PEs: vertex x belongs to tile x / B; an edge is local when both ends
// are in one tile, a cut edge otherwise.

// Runs of equal keys among the lanes of a warp (key 0xffffffff = no item):
// returns the lane mask of this lane's run and the run's first lane.  Inputs
// grouped by tile give long runs, so one atomic per run serves the whole run.
__device__ __forceinline__ uint32_t warp_run(uint32_t key, int &head_lane) {
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
  const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
  head_lane = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));   // last head at or below this lane
  const uint32_t above = heads & ~(0xffffffffu >> (31 - lane));    // heads above this lane
  const int next = above ? __ffs(above) - 1 : 32;
  return (next >= 32 ? 0xffffffffu : ((1u << next) - 1u)) & ~((1u << head_lane) - 1u);
}

// Pass over the input: vertex-range check, per-vertex minimum key over incident
// cut edges (cutmin), number of local edges per tile, total local edges, and
// the largest weight (key layout).  Local-edge counts are aggregated per warp.
__global__ void __launch_bounds__(BLOCK) tile_count_kernel(EdgeList in, uint64_t m, uint32_t n, uint32_t B,
                                                           u64 *cutmin, uint32_t *count, u64 *local_total,
                                                           uint32_t *max_w, uint32_t *err) {
  const uint64_t ntiles = (m + TILE - 1) / TILE;
  uint32_t nlocal = 0, mx = 0;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t tb = tile * TILE;
    uint32_t eu[ITEMS], ev[ITEMS], ew[ITEMS];
    if (tb + TILE <= m && aligned16_dev(in.u) && aligned16_dev(in.v) && aligned16_dev(in.w)) {
      load_striped(in.u, tb, eu);
      load_striped(in.v, tb, ev);
      load_striped(in.w, tb, ew);
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const uint64_t j = tb + item_off(k);
        eu[k] = j < m ? __ldg(in.u + j) : 0u;
        ev[k] = j < m ? __ldg(in.v + j) : 0u;
        ew[k] = j < m ? __ldg(in.w + j) : 0u;
      }
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint64_t j = tb + item_off(k);
      bool ok = j < m;
      if (ok && (eu[k] >= n || ev[k] >= n)) {
        atomicOr(err, ERR_VERTEX);
        ok = false;
      }
      if (ok) mx = max(mx, ew[k]);
      ok = ok && eu[k] != ev[k];
      const uint32_t tu = eu[k] / B, tv = ev[k] / B;
      const bool local = ok && tu == tv;
      int head;
      const uint32_t run = warp_run(local ? tu : 0xffffffffu, head);
      if (local && (threadIdx.x & 31) == (unsigned)head) atomicAdd(count + tu, (uint32_t)__popc(run));
      nlocal += local ? 1u : 0u;
      if (ok && !local) {
        const u64 key = edge_key(ew[k], (uint32_t)j);
        if (key < __ldca(cutmin + eu[k])) atomicMin(cutmin + eu[k], key);
        if (key < __ldca(cutmin + ev[k])) atomicMin(cutmin + ev[k], key);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nlocal += __shfl_xor_sync(0xffffffffu, nlocal, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (nlocal) atomicAdd(local_total, (u64)nlocal);
    if (mx > __ldca(max_w)) atomicMax(max_w, mx);
  }
}

// Exclusive scan of the per-tile counts into offsets[0..ntiles] (one block).
__global__ void __launch_bounds__(1024) tile_scan_kernel(const uint32_t *count, uint32_t ntiles, u64 *offsets) {
  __shared__ u64 s_w[33];
  __shared__ u64 s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < ntiles; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const u64 x = i < ntiles ? count[i] : 0;
    u64 incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const u64 v = s_w[lane];
      u64 wi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_w[lane] = wi - v;
      if (lane == 31) s_w[32] = wi;
    }
    __syncthreads();
    const u64 carry = s_carry;
    if (i < ntiles) offsets[i] = carry + s_w[wid] + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_w[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[ntiles] = s_carry;
}

// Scatters the local edges into per-tile buckets: packed tile-local ends
// (u | v << 16), weight and id.  Order inside a bucket is unspecified.  The
// cut edges (ends in different tiles) go to an edge list with their input ids,
// in unspecified order; *cut_fill counts them (zero before the launch).
__global__ void __launch_bounds__(BLOCK) tile_scatter_kernel(EdgeList in, uint64_t m, uint32_t n, uint32_t B,
                                                             const u64 *offsets, uint32_t *fill, uint32_t *b_ends,
                                                             uint32_t *b_w, uint32_t *b_id, EdgeOut cut,
                                                             u64 *cut_fill) {
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  __shared__ u64 s_base;
  const uint64_t ntiles = (m + TILE - 1) / TILE;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t tb = tile * TILE;
    uint32_t eu[ITEMS], ev[ITEMS], ew[ITEMS];
    if (tb + TILE <= m && aligned16_dev(in.u) && aligned16_dev(in.v) && aligned16_dev(in.w)) {
      load_striped(in.u, tb, eu);
      load_striped(in.v, tb, ev);
      load_striped(in.w, tb, ew);
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const uint64_t j = tb + item_off(k);
        eu[k] = j < m ? __ldg(in.u + j) : 0u;
        ev[k] = j < m ? __ldg(in.v + j) : 0u;
        ew[k] = j < m ? __ldg(in.w + j) : 0u;
      }
    }
    uint32_t is_cut = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint64_t j = tb + item_off(k);
      const bool ok = j < m && eu[k] < n && ev[k] < n && eu[k] != ev[k];
      const uint32_t tu = eu[k] / B, tv = ev[k] / B;
      const bool local = ok && tu == tv;
      if (ok && !local) is_cut |= 1u << k;
      int head;
      const uint32_t run = warp_run(local ? tu : 0xffffffffu, head);
      uint32_t pos = 0;
      if (local && (threadIdx.x & 31) == (unsigned)head) pos = atomicAdd(fill + tu, (uint32_t)__popc(run));
      pos = __shfl_sync(0xffffffffu, pos, head);
      if (local) {
        const u64 at = offsets[tu] + pos + ((threadIdx.x & 31) - (uint32_t)head);
        b_ends[at] = (eu[k] - tu * B) | ((ev[k] - tu * B) << 16);
        b_w[at] = ew[k];
        b_id[at] = (uint32_t)j;
      }
    }
    // one claim per tile for its cut edges
    uint32_t total;
    uint32_t at = block_exclusive_scan((uint32_t)__popc(is_cut), total, s_warp);
    if (threadIdx.x == 0) s_base = total ? atomicAdd(cut_fill, (u64)total) : 0;
    __syncthreads();
    const u64 base = s_base;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (is_cut >> k & 1u) {
        cut.u[base + at] = eu[k];
        cut.v[base + at] = ev[k];
        cut.w[base + at] = ew[k];
        cut.id[base + at] = (uint32_t)(tb + item_off(k));
        ++at;
      }
    }
    __syncthreads();  // s_base and s_warp are reused by the next tile
  }
}

// One block per tile: synchronous Borůvka rounds on the tile's local edges in
// shared memory.  A component hooks along its lightest local edge only when
// that edge is lighter than every cut edge incident to the component (then it
// is the component's lightest edge overall, an MSF edge by the cut property);
// 2-cycles keep the smaller vertex as root.  Rounds repeat until no component
// hooks.  Writes the tile root of every vertex to parent[] and sets the bits
// of the contracted edges.  A tile whose edges exceed the shared-memory
// capacity runs the same rounds reading its bucket from global memory.
constexpr int TC_THREADS = 512;
constexpr int TC_EPT = 16;  // edges per thread in the in-place compaction (capacity TC_EPT * TC_THREADS)

__device__ __forceinline__ uint32_t tc_exclusive_scan(uint32_t x, uint32_t &total, uint32_t *s_warp) {
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
    const uint32_t wv = lane < TC_THREADS / 32 ? s_warp[lane] : 0u;
    uint32_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < TC_THREADS / 32) s_warp[lane] = wi - wv;
    if (lane == TC_THREADS / 32 - 1) s_warp[TC_THREADS / 32] = wi;
  }
  __syncthreads();
  total = s_warp[TC_THREADS / 32];
  return s_warp[wid] + incl - x;
}

__global__ void __launch_bounds__(TC_THREADS, 2) tile_contract_kernel(uint32_t n, uint32_t B, const u64 *cutmin,
                                                                    const u64 *offsets, const uint32_t *b_ends,
                                                                    const uint32_t *b_w, const uint32_t *b_id,
                                                                    uint32_t edge_cap, uint32_t *parent,
                                                                    uint32_t *bits, EdgeOut rest, u64 *rest_fill,
                                                                    uint32_t *err, int filter_heavy, u64 *wsum) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  u64 *best = reinterpret_cast<u64 *>(smem_dyn);  // [B]
  u64 *comp = best + B;                           // [B] component cut minimum (valid at roots)
  u64 *skey = comp + B;                           // [edge_cap]
  uint32_t *lab = reinterpret_cast<uint32_t *>(skey + edge_cap);  // [B]
  uint32_t *hook = lab + B;                                        // [B]
  uint32_t *other = hook + B;                                      // [B]
  uint32_t *sends = other + B;                                     // [edge_cap]
  __shared__ uint32_t s_any, s_ne, s_light, s_warp[TC_THREADS / 32 + 1];
  __shared__ u64 s_base, s_pivot;

  const uint32_t t = blockIdx.x;
  const uint64_t vbase = (uint64_t)t * B;
  const uint32_t nv = (uint32_t)min((uint64_t)B, (uint64_t)n - vbase);
  const u64 e0 = offsets[t];
  const uint32_t ne0 = (uint32_t)(offsets[t + 1] - e0);
  __shared__ unsigned long long s_wsum;  // weights of the edges this block's components chose
  if (threadIdx.x == 0) s_wsum = 0;
  // In shared memory the edges hold the labels of their ends' components and
  // are compacted after every round (edges inside a component are dropped);
  // from global memory they are read as input ends and mapped through lab[].
  const bool in_smem = ne0 <= edge_cap;
  for (uint32_t x = threadIdx.x; x < nv; x += TC_THREADS) {
    lab[x] = x;
    comp[x] = cutmin[vbase + x];
  }
  if (in_smem) {
    for (uint32_t e = threadIdx.x; e < ne0; e += TC_THREADS) {
      sends[e] = b_ends[e0 + e];
      skey[e] = edge_key(b_w[e0 + e], b_id[e0 + e]);
    }
  }
  if (threadIdx.x == 0) s_ne = ne0;
  __syncthreads();
  // Recursive filtering inside the tile (the Filter-Borůvka idea applied to
  // local preprocessing, Section 6.2): the rounds first use only the light
  // edges (key <= the median of 32 evenly spaced keys); the heavy ones are
  // relabelled with them and the compaction drops those that fall inside a
  // component (the filter).  When the light edges no longer hook, every edge
  // takes part.  A light edge is lighter than every heavy one, so the hooking
  // rule (lightest incident edge, below the cut minimum) is unchanged.
  if (threadIdx.x < 32) {
    const uint32_t lane = threadIdx.x;
    const bool on = filter_heavy && in_smem && ne0 >= 64;
    u64 v = on ? skey[(uint32_t)(((uint64_t)lane * ne0) / 32)] : 0ULL;
    for (uint32_t k = 2; k <= 32; k <<= 1)  // bitonic sort of the warp's 32 keys, ascending
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        const u64 o = __shfl_xor_sync(0xffffffffu, v, j);
        v = (((lane & j) == 0) == ((lane & k) == 0)) ? (o < v ? o : v) : (o > v ? o : v);
      }
    const u64 med = __shfl_sync(0xffffffffu, v, 15);
    if (lane == 0) {
      s_light = on ? 1u : 0u;
      s_pivot = on ? med : KEY_INF;
    }
  }
  __syncthreads();
  for (uint32_t round = 0; round <= 2 * nv + 2; ++round) {
    const uint32_t ne = s_ne;
    const u64 lim = s_light ? s_pivot : KEY_INF;  // edges above it wait for the second phase
    for (uint32_t c = threadIdx.x; c < nv; c += TC_THREADS) best[c] = KEY_INF;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < ne; e += TC_THREADS) {  // lightest local edge per component
      const uint32_t pe = in_smem ? sends[e] : b_ends[e0 + e];
      const u64 k = in_smem ? skey[e] : edge_key(b_w[e0 + e], b_id[e0 + e]);
      const uint32_t a = in_smem ? (pe & 0xffffu) : lab[pe & 0xffffu], b = in_smem ? (pe >> 16) : lab[pe >> 16];
      if (a != b && k <= lim) {
        if (k < best[a]) atomicMin(best + a, k);
        if (k < best[b]) atomicMin(best + b, k);
      }
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < nv; c += TC_THREADS)  // hook only below every incident cut edge
      if (lab[c] != c || !(best[c] < comp[c])) best[c] = KEY_INF;
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < ne; e += TC_THREADS) {  // far end of each hooking component's edge
      const uint32_t pe = in_smem ? sends[e] : b_ends[e0 + e];
      const u64 k = in_smem ? skey[e] : edge_key(b_w[e0 + e], b_id[e0 + e]);
      const uint32_t a = in_smem ? (pe & 0xffffu) : lab[pe & 0xffffu], b = in_smem ? (pe >> 16) : lab[pe >> 16];
      if (a != b && k <= lim) {
        if (best[a] == k) other[a] = b;
        if (best[b] == k) other[b] = a;
      }
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < nv; c += TC_THREADS) {
      hook[c] = c;
      if (best[c] != KEY_INF) {
        const uint32_t o = other[c];
        const bool root = best[o] == best[c] && c < o;
        if (!root) {
          hook[c] = o;
          const uint32_t id = (uint32_t)best[c];
          atomicOr(bits + (id >> 5), 1u << (id & 31));
          atomicAdd(&s_wsum, (unsigned long long)(best[c] >> 32));
          s_any = 1;
        }
      }
    }
    __syncthreads();
    if (!s_any) {
      if (!s_light) break;
      __syncthreads();  // every thread has read s_light
      if (threadIdx.x == 0) s_light = 0;
      __syncthreads();
      continue;  // the heavy edges left join the rounds
    }
    // every component of the last round follows its hooks to the new root
    // (the hooks form a forest: at most nv steps)
    for (uint32_t c = threadIdx.x; c < nv; c += TC_THREADS) {
      if (lab[c] != c) continue;
      uint32_t r = c;
      for (uint32_t step = 0; step <= nv; ++step) {
        const uint32_t h = hook[r];
        if (h == r) break;
        r = h;
        if (step == nv) atomicOr(err, ERR_JUMP);
      }
      other[c] = r;
    }
    __syncthreads();
    // merge the cut minima into the new roots, relabel the vertices
    for (uint32_t c = threadIdx.x; c < nv; c += TC_THREADS) {
      const uint32_t l = lab[c];
      const uint32_t r = other[l];
      if (l == c && r != c) atomicMin(comp + r, comp[c]);
      lab[c] = r;
    }
    if (in_smem) {  // relabel the edges to the new roots and keep those between components
      uint32_t pe[TC_EPT];
      u64 k[TC_EPT];
      uint32_t keep = 0, cnt = 0;
#pragma unroll
      for (int i = 0; i < TC_EPT; ++i) {
        const uint32_t e = threadIdx.x + (uint32_t)i * TC_THREADS;
        pe[i] = 0;
        k[i] = 0;
        if (e < ne) {
          const uint32_t x = sends[e];
          const uint32_t a = other[x & 0xffffu], b = other[x >> 16];
          pe[i] = a | (b << 16);
          k[i] = skey[e];
          if (a != b) {
            keep |= 1u << i;
            ++cnt;
          }
        }
      }
      uint32_t total;
      uint32_t pos = tc_exclusive_scan(cnt, total, s_warp);  // all reads precede its barriers
#pragma unroll
      for (int i = 0; i < TC_EPT; ++i) {
        if (keep >> i & 1u) {
          sends[pos] = pe[i];
          skey[pos] = k[i];
          ++pos;
        }
      }
      if (threadIdx.x == 0) s_ne = total;
    }
    __syncthreads();
  }
  // every hook step ends in a barrier, so the block's sum of chosen weights is complete
  if (threadIdx.x == 0 && wsum && s_wsum)
    atomicAdd(reinterpret_cast<unsigned long long *>(wsum) + (t & (WSUM_SLOTS - 1)), s_wsum);
  for (uint32_t x = threadIdx.x; x < nv; x += TC_THREADS) parent[vbase + x] = (uint32_t)(vbase + lab[x]);
  // The local edges left between different components of the tile join the
  // cut edges in the contracted graph, with their ends at the tile roots.
  if (in_smem) {
    const uint32_t ne = s_ne;
    if (threadIdx.x == 0) s_base = ne ? atomicAdd(rest_fill, (u64)ne) : 0;
    __syncthreads();
    const u64 base = s_base;
    for (uint32_t e = threadIdx.x; e < ne; e += TC_THREADS) {
      const uint32_t pe = sends[e];
      const u64 k = skey[e];
      rest.u[base + e] = (uint32_t)(vbase + (pe & 0xffffu));
      rest.v[base + e] = (uint32_t)(vbase + (pe >> 16));
      rest.w[base + e] = (uint32_t)(k >> 32);
      rest.id[base + e] = (uint32_t)k;
    }
  } else {
    const int lane = threadIdx.x & 31;
    for (uint32_t b0 = 0; b0 < ne0; b0 += TC_THREADS) {
      const uint32_t e = b0 + threadIdx.x;
      uint32_t a = 0, b = 0;
      if (e < ne0) {
        const uint32_t pe = b_ends[e0 + e];
        a = lab[pe & 0xffffu];
        b = lab[pe >> 16];
      }
      const bool keep = e < ne0 && a != b;
      const uint32_t kb = __ballot_sync(0xffffffffu, keep);
      if (!kb) continue;
      const int lead = __ffs(kb) - 1;
      u64 base = 0;
      if (lane == lead) base = atomicAdd(rest_fill, (u64)__popc(kb));
      base = __shfl_sync(0xffffffffu, base, lead);
      if (keep) {
        const u64 at = base + __popc(kb & ((1u << lane) - 1u));
        rest.u[at] = (uint32_t)(vbase + a);
        rest.v[at] = (uint32_t)(vbase + b);
        rest.w[at] = b_w[e0 + e];
        rest.id[at] = b_id[e0 + e];
      }
    }
  }
}

// ---------------------------------------------------------- radix sort

// Stable LSD radix sort of (u64 key, u32 value) pairs, 8-bit digits, for the
// sort-based parallel-edge removal.  Each of RS_BLOCKS blocks owns one
// contiguous chunk of the input: per pass it counts its chunk's digits, one
// block scans the counts (digit-major, so a digit's items from earlier chunks
// come first), and each block scatters its chunk in input order.  Within a
// 2048-item tile the items go in eight sub-rounds of 256 consecutive items; a
// warp ranks equal digits among its lanes with __match_any_sync, and the
// per-warp counts of a sub-round are scanned in warp order: the result is
// stable.
constexpr int RS_BITS = 8, RS_BINS = 1 << RS_BITS, RS_WARPS = BLOCK / 32;

__device__ __forceinline__ void rs_chunk(uint64_t m, uint64_t &lo, uint64_t &hi) {
  const uint64_t per = ((m + gridDim.x - 1) / gridDim.x + TILE - 1) / TILE * TILE;
  lo = min(m, (uint64_t)blockIdx.x * per);
  hi = min(m, lo + per);
}

__global__ void __launch_bounds__(BLOCK) radix_hist_kernel(const u64 *keys, uint64_t m, int shift, uint32_t *hist) {
  __shared__ uint32_t sh[RS_BINS];
  for (int d = threadIdx.x; d < RS_BINS; d += BLOCK) sh[d] = 0;
  __syncthreads();
  uint64_t lo, hi;
  rs_chunk(m, lo, hi);
  for (uint64_t i = lo + threadIdx.x; i < hi; i += BLOCK) atomicAdd(&sh[(keys[i] >> shift) & (RS_BINS - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += BLOCK) hist[(uint64_t)d * gridDim.x + blockIdx.x] = sh[d];
}

// Exclusive scan, in place, of `count` entries (one block of 1024 threads).
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *a, uint32_t count) {
  __shared__ uint32_t s_w[33];
  const uint32_t per = (count + 1023) / 1024;
  const uint32_t lo = min(count, threadIdx.x * per), hi = min(count, lo + per);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += a[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const uint32_t v = s_w[lane];
    uint32_t wi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    s_w[lane] = wi - v;
  }
  __syncthreads();
  uint32_t run = s_w[wid] + incl - sum;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t x = a[i];
    a[i] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(BLOCK) radix_scatter_kernel(const u64 *keys, const uint32_t *vals, uint64_t m,
                                                              int shift, const uint32_t *offsets, u64 *keys_out,
                                                              uint32_t *vals_out) {
  __shared__ uint32_t base[RS_BINS];
  __shared__ uint32_t wc[RS_WARPS][RS_BINS];
  for (int d = threadIdx.x; d < RS_BINS; d += BLOCK) base[d] = offsets[(uint64_t)d * gridDim.x + blockIdx.x];
  uint64_t lo, hi;
  rs_chunk(m, lo, hi);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (uint64_t tb = lo; tb < hi; tb += BLOCK) {  // one sub-round: BLOCK consecutive items
    const uint64_t i = tb + threadIdx.x;
    const bool in = i < hi;
    const u64 k = in ? keys[i] : 0;
    const uint32_t val = in ? vals[i] : 0u;
    const uint32_t d = in ? (uint32_t)((k >> shift) & (RS_BINS - 1)) : (uint32_t)RS_BINS;
    for (int w = 0; w < RS_WARPS; ++w) wc[w][threadIdx.x & (RS_BINS - 1)] = 0;
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (in && rank == 0) wc[wid][d] = __popc(peers);
    __syncthreads();
    {  // warp-order exclusive offsets of each digit (thread t owns digit t)
      const int dd = threadIdx.x;
      uint32_t run = base[dd];
      for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = wc[w][dd];
        wc[w][dd] = run;
        run += c;
      }
      base[dd] = run;
    }
    __syncthreads();
    if (in) {
      const uint32_t pos = wc[wid][d] + rank;
      keys_out[pos] = k;
      vals_out[pos] = val;
    }
    __syncthreads();
  }
}

// Exclusive scan of the digit counts in three coalesced steps: per-segment
// sums, a scan of the (few) sums, per-segment scans from their offsets.
constexpr uint32_t RS_SEG = 4096;

__global__ void __launch_bounds__(BLOCK) rs_seg_sum_kernel(const uint32_t *a, uint32_t count, uint32_t *sums) {
  __shared__ uint32_t s_w[BLOCK / 32];
  const uint32_t lo = blockIdx.x * RS_SEG, hi = min(count, lo + RS_SEG);
  uint32_t x = 0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += BLOCK) x += a[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < BLOCK / 32; ++w) t += s_w[w];
    sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(BLOCK) rs_seg_scan_kernel(uint32_t *a, uint32_t count, const uint32_t *offs) {
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  const uint32_t lo = blockIdx.x * RS_SEG, hi = min(count, lo + RS_SEG);
  uint32_t carry = offs[blockIdx.x];
  for (uint32_t b0 = lo; b0 < hi; b0 += BLOCK) {  // uniform trip count
    const uint32_t i = b0 + threadIdx.x;
    const uint32_t x = i < hi ? a[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(x, total, s_warp);
    if (i < hi) a[i] = carry + ex;
    carry += total;
    __syncthreads();  // s_warp is reused by the next chunk
  }
}

int radix_blocks(uint64_t m, int sms) {
  const uint64_t tiles = (m + TILE - 1) / TILE;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)sms * 4));
}

size_t radix_hist_bytes(uint64_t m, int sms) {
  const size_t entries = (size_t)RS_BINS * radix_blocks(m, sms);
  return (entries + (entries + RS_SEG - 1) / RS_SEG) * sizeof(uint32_t);  // counts, then segment sums
}

bool launch_radix_sort(u64 *keys, uint32_t *vals, u64 *keys_tmp, uint32_t *vals_tmp, uint64_t m, int bits,
                       uint32_t *hist, int sms, cudaStream_t s) {
  if (m == 0) return false;
  const int nb = radix_blocks(m, sms);
  const uint32_t entries = (uint32_t)RS_BINS * (uint32_t)nb;
  bool swapped = false;
  for (int shift = 0; shift < bits; shift += RS_BITS) {
    const u64 *ki = swapped ? keys_tmp : keys;
    const uint32_t *vi = swapped ? vals_tmp : vals;
    u64 *ko = swapped ? keys : keys_tmp;
    uint32_t *vo = swapped ? vals : vals_tmp;
    radix_hist_kernel<<<nb, BLOCK, 0, s>>>(ki, m, shift, hist);
    const uint32_t nseg = (entries + RS_SEG - 1) / RS_SEG;  // <= 1024: one block scans the segment sums
    uint32_t *sums = hist + entries;
    rs_seg_sum_kernel<<<nseg, BLOCK, 0, s>>>(hist, entries, sums);
    radix_scan_kernel<<<1, 1024, 0, s>>>(sums, nseg);
    rs_seg_scan_kernel<<<nseg, BLOCK, 0, s>>>(hist, entries, sums);
    radix_scatter_kernel<<<nb, BLOCK, 0, s>>>(ki, vi, m, shift, hist, ko, vo);
    swapped = !swapped;
  }
  return swapped;
}

// ------------------------------------------- sort-based parallel-edge removal

// Parallel-edge removal by sorting (Section 2.3; the sort variant of Section
// 4.3): sort the list by (w, id), then stably by the unordered pair
// {min(u,v), max(u,v)}; the first edge of every pair run is the pair's lightest.
__global__ void sd_key_kernel(EdgeList T, uint64_t m, int ib, u64 *keys, uint32_t *vals) {
  for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < m; j += (uint64_t)gridDim.x * BLOCK) {
    keys[j] = ((u64)T.w[j] << ib) | (u64)T.id[j];
    vals[j] = (uint32_t)j;
  }
}

__global__ void sd_pair_kernel(EdgeList T, const uint32_t *idx, uint64_t m, int vb, u64 *keys, uint32_t *vals) {
  for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < m; j += (uint64_t)gridDim.x * BLOCK) {
    const uint32_t i = idx[j];
    const uint32_t u = T.u[i], v = T.v[i];
    keys[j] = ((u64)min(u, v) << vb) | (u64)max(u, v);
    vals[j] = i;
  }
}

// Keeps position j of the pair-sorted order when it starts a run, gathers that
// edge from T and emits it like a compaction (relaxing best[] / recording ends).
__global__ void __launch_bounds__(BLOCK) sd_emit_kernel(const u64 *pk, const uint32_t *idx, uint64_t m, CompactArgs a) {
  __shared__ uint32_t s_u[TILE], s_v[TILE], s_w[TILE], s_id[TILE];
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  __shared__ uint32_t s_base[1];
  const uint64_t tb = (uint64_t)blockIdx.x * TILE;
  if (tb >= m) return;
  uint32_t eu[ITEMS], ev[ITEMS], ew[ITEMS], ei[ITEMS];
  uint32_t keep = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint64_t j = tb + item_off(k);
    const bool head = j < m && (j == 0 || pk[j] != pk[j - 1]);
    eu[k] = ev[k] = ew[k] = ei[k] = 0;
    if (head) {
      const uint32_t i = idx[j];
      eu[k] = a.in.u[i];
      ev[k] = a.in.v[i];
      ew[k] = a.in.w[i];
      ei[k] = a.in.id[i];
      if (eu[k] != ev[k]) keep |= 1u << k;  // self-loops are never kept
    }
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan((uint32_t)__popc(keep), total, s_warp);
  const uint64_t obase = tile_claim(a.st.total, total, s_base);
  emit_survivors<BLOCK, ITEMS>(a, keep, excl, total, obase, eu, ev, ew, ei, s_u, s_v, s_w, s_id);
}

size_t sort_dedupe_scratch_bytes(uint64_t m, int sms) {
  return 2 * ((m * 8 + 255) / 256 * 256) + 2 * ((m * 4 + 255) / 256 * 256) + radix_hist_bytes(m, sms) + 256;
}

void launch_sort_dedupe(EdgeList T, uint64_t m, int vbits, int wbits, int ibits, const CompactArgs &emit,
                        void *scratch, int sms, cudaStream_t s) {
  if (m == 0) return;
  char *p = (char *)scratch;
  const size_t kb = (m * 8 + 255) / 256 * 256, vb = (m * 4 + 255) / 256 * 256;
  u64 *k0 = (u64 *)p, *k1 = (u64 *)(p + kb);
  uint32_t *v0 = (uint32_t *)(p + 2 * kb), *v1 = (uint32_t *)(p + 2 * kb + vb);
  uint32_t *hist = (uint32_t *)(p + 2 * kb + 2 * vb);
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((m + BLOCK - 1) / BLOCK, (uint64_t)sms * 8));
  sd_key_kernel<<<grid, BLOCK, 0, s>>>(T, m, ibits, k0, v0);
  const bool in1 = launch_radix_sort(k0, v0, k1, v1, m, wbits + ibits, hist, sms, s);
  u64 *ka = in1 ? k1 : k0, *kb2 = in1 ? k0 : k1;
  uint32_t *va = in1 ? v1 : v0, *vb2 = in1 ? v0 : v1;
  sd_pair_kernel<<<grid, BLOCK, 0, s>>>(T, va, m, vbits, kb2, vb2);  // pairs in (w, id) order
  const bool in2 = launch_radix_sort(kb2, vb2, ka, va, m, 2 * vbits, hist, sms, s);
  const u64 *pk = in2 ? ka : kb2;
  const uint32_t *pidx = in2 ? va : vb2;
  sd_emit_kernel<<<(unsigned)((m + TILE - 1) / TILE), BLOCK, 0, s>>>(pk, pidx, m, emit);
}

// ----------------------------------------------- sort-based minEdges

// minEdges as a segmented minimum (the sorted-edge representation of Sections
// 2.2 and 4.5): both ends of every edge become (vertex, 2j + side) entries,
// sorted by vertex; each run of equal vertices is reduced by warp-segmented
// minima with one atomic per run and warp, instead of one per edge end.
__global__ void me_ends_kernel(EdgeList E, uint64_t m, uint32_t n, int validate, u64 *keys, uint32_t *vals,
                               uint32_t *err) {
  for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < m; j += (uint64_t)gridDim.x * BLOCK) {
    uint32_t u = E.u[j], v = E.v[j];
    if (validate && (u >= n || v >= n)) {
      atomicOr(err, ERR_VERTEX);
      u = v = 0;  // dropped below as a self-loop
    }
    const bool live = u != v;
    keys[2 * j] = live ? u : n;  // dead entries sort last (key n, above every vertex)
    keys[2 * j + 1] = live ? v : n;
    vals[2 * j] = (uint32_t)(2 * j);
    vals[2 * j + 1] = (uint32_t)(2 * j + 1);
  }
}

__global__ void me_segmin_kernel(const u64 *keys, const uint32_t *vals, uint64_t entries, uint32_t n, EdgeList E,
                                 KeyLayout kl, u64 *best) {
  const int lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
  for (uint64_t b0 = (uint64_t)blockIdx.x * BLOCK; b0 < entries; b0 += stride) {  // warp-uniform trip count
    const uint64_t p = b0 + threadIdx.x;
    uint32_t vtx = 0xffffffffu;
    u64 rk = KEY_INF;
    if (p < entries && keys[p] < n) {
      vtx = (uint32_t)keys[p];
      const uint32_t e = vals[p] >> 1, side = vals[p] & 1u;
      const uint32_t other = side ? E.u[e] : E.v[e];
      rk = relax_key(kl, E.w[e], E.id ? E.id[e] : e, other);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {  // segmented minimum over runs of one vertex
      const u64 pr = __shfl_up_sync(0xffffffffu, rk, o);
      const uint32_t pv = __shfl_up_sync(0xffffffffu, vtx, o);
      if (lane >= o && pv == vtx && pr < rk) rk = pr;
    }
    const uint32_t nv = __shfl_down_sync(0xffffffffu, vtx, 1);
    if (vtx != 0xffffffffu && (lane == 31 || nv != vtx) && rk < __ldca(best + vtx)) atomicMin(best + vtx, rk);
  }
}

size_t min_edges_sort_scratch_bytes(uint64_t m, int sms) {
  const uint64_t e = 2 * m;
  return 2 * ((e * 8 + 255) / 256 * 256) + 2 * ((e * 4 + 255) / 256 * 256) + radix_hist_bytes(e, sms) + 256;
}

bool launch_min_edges_sort(EdgeList E, uint64_t m, uint32_t n, int validate, KeyLayout kl, u64 *best, uint32_t *err,
                           void *scratch, int sms, cudaStream_t s) {
  if (m == 0) return true;
  if (2 * m >= (1ULL << 32)) return false;  // entry values are 32-bit
  const uint64_t e = 2 * m;
  char *p = (char *)scratch;
  const size_t kb = (e * 8 + 255) / 256 * 256, vb = (e * 4 + 255) / 256 * 256;
  u64 *k0 = (u64 *)p, *k1 = (u64 *)(p + kb);
  uint32_t *v0 = (uint32_t *)(p + 2 * kb), *v1 = (uint32_t *)(p + 2 * kb + vb);
  uint32_t *hist = (uint32_t *)(p + 2 * kb + 2 * vb);
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((m + BLOCK - 1) / BLOCK, (uint64_t)sms * 8));
  me_ends_kernel<<<grid, BLOCK, 0, s>>>(E, m, n, validate, k0, v0, err);
  int bits = 1;
  while (bits < 33 && (1ULL << bits) <= (uint64_t)n) ++bits;  // keys 0..n (n: dead entries)
  const bool in1 = launch_radix_sort(k0, v0, k1, v1, e, bits, hist, sms, s);
  const unsigned g2 = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((e + BLOCK - 1) / BLOCK, (uint64_t)sms * 8));
  me_segmin_kernel<<<g2, BLOCK, 0, s>>>(in1 ? k1 : k0, in1 ? v1 : v0, e, n, E, kl, best);
  return true;
}

// ------------------------------------------------- device-driven round loop

// State of the Borůvka rounds run as a CUDA graph: a conditional WHILE node
// repeats a body of two rounds (lists and active lists alternate between slot
// 0 and slot 1) while round_cond_kernel sets its condition.  Counts live here,
// so no round waits for the host.
__global__ void round_init_kernel(GraphRounds *g, uint64_t m, uint64_t n_act) {
  g->ce[0] = m;
  g->ca[0] = n_act;
  g->ce[1] = g->ca[1] = 0;  // outputs of the first round
  g->jflag = 0;
  g->iter = 0;
  g->reason = ROUNDS_RUNNING;
  g->slot = 0;
  g->saved_ce = g->saved_ca = 0;
}

// The same from a device count of edges; the active count is filled by the
// hooking launch of the call's first round, which runs before the graph.
__global__ void round_init_dev_kernel(GraphRounds *g, const u64 *m_dev, uint64_t cap) {
  g->ce[0] = min((uint64_t)*m_dev, cap);
  g->ca[0] = 0;
  g->ce[1] = g->ca[1] = 0;
  g->jflag = 0;
  g->iter = 0;
  g->reason = ROUNDS_RUNNING;
  g->slot = 0;
  g->saved_ce = g->saved_ca = 0;
}

// The graph's first node: run the loop only if there are active vertices and
// edges and the jump before the graph reached the roots.  Otherwise end here
// and publish the outcome as round_cond_kernel does.
__global__ void round_pre_kernel(GraphRounds *g, cudaGraphConditionalHandle h, u64 *out_counts, uint32_t *err_handback) {
  unsigned int go = 0;
  if (g->jflag) {
    g->reason = ROUNDS_JUMP;
    if (err_handback) atomicOr(err_handback, ERR_HANDBACK);
  } else if (g->ca[0] == 0 || g->ce[0] == 0) {
    g->reason = ROUNDS_DONE;
  } else {
    go = 1;
  }
  if (!go) {
    g->slot = 0;
    g->saved_ce = g->ce[0];
    g->saved_ca = g->ca[0];
    out_counts[0] = g->saved_ce;
    out_counts[1] = g->saved_ca;
    out_counts[2] = (u64)g->reason;
  }
  g->jflag = 0;
  cudaGraphSetConditional(h, go);
}

// After the first round of the body (slot 0 -> 1): stop early (the second
// round then sees zero counts and does nothing) when the jump did not reach
// the roots or the base case fits.
__global__ void round_check_kernel(GraphRounds *g, int base_ok, uint32_t *err_handback) {
  if (g->jflag || (base_ok && g->ca[1] > 0 && g->ca[1] <= BASE_MAX_N && g->ce[1] > 0 && g->ce[1] <= BASE_MAX_M)) {
    if (g->jflag && err_handback) atomicOr(err_handback, ERR_HANDBACK);
    g->reason = g->jflag ? ROUNDS_JUMP : ROUNDS_BASE;
    g->slot = 1;
    g->saved_ce = g->ce[1];
    g->saved_ca = g->ca[1];
    g->ce[1] = g->ca[1] = 0;
  }
  g->ce[0] = g->ca[0] = 0;  // outputs of the second round
  g->jflag = 0;
}

// After the second round (slot 1 -> 0): decide whether the body runs again,
// and publish the outcome in the solver's counters (edges, active, info).
__global__ void round_cond_kernel(GraphRounds *g, cudaGraphConditionalHandle h, int base_ok, uint32_t max_iter,
                                  u64 *out_counts, uint32_t *err_handback) {
  const uint32_t it = ++g->iter;
  unsigned int go = 0;
  if (g->reason == ROUNDS_RUNNING) {
    if (g->jflag) {
      g->reason = ROUNDS_JUMP;
    } else if (g->ca[0] == 0 || g->ce[0] == 0) {
      g->reason = ROUNDS_DONE;
    } else if (base_ok && g->ca[0] <= BASE_MAX_N && g->ce[0] <= BASE_MAX_M) {
      g->reason = ROUNDS_BASE;
    } else if (it >= max_iter) {
      g->reason = ROUNDS_BOUND;
    } else {
      go = 1;
    }
    if (!go) {
      g->slot = 0;
      g->saved_ce = g->ce[0];
      g->saved_ca = g->ca[0];
      if (err_handback && (g->reason == ROUNDS_JUMP || g->reason == ROUNDS_BOUND)) atomicOr(err_handback, ERR_HANDBACK);
    }
  }
  out_counts[0] = g->saved_ce;
  out_counts[1] = g->saved_ca;
  out_counts[2] = (u64)g->reason | ((u64)g->slot << 8) | ((u64)it << 16);
  g->ce[1] = g->ca[1] = 0;  // outputs of the next body's first round
  g->jflag = 0;
  cudaGraphSetConditional(h, go);
}

void launch_round_init(GraphRounds *g, uint64_t m, uint64_t n_act, cudaStream_t s) {
  round_init_kernel<<<1, 1, 0, s>>>(g, m, n_act);
}
void launch_round_init_dev(GraphRounds *g, const u64 *m_dev, uint64_t cap, cudaStream_t s) {
  round_init_dev_kernel<<<1, 1, 0, s>>>(g, m_dev, cap);
}
void launch_round_pre(GraphRounds *g, cudaGraphConditionalHandle h, u64 *out_counts, uint32_t *err_handback,
                      cudaStream_t s) {
  round_pre_kernel<<<1, 1, 0, s>>>(g, h, out_counts, err_handback);
}
void launch_round_check(GraphRounds *g, int base_ok, uint32_t *err_handback, cudaStream_t s) {
  round_check_kernel<<<1, 1, 0, s>>>(g, base_ok, err_handback);
}
void launch_round_cond(GraphRounds *g, cudaGraphConditionalHandle h, int base_ok, uint32_t max_iter, u64 *out_counts,
                       uint32_t *err_handback, cudaStream_t s) {
  round_cond_kernel<<<1, 1, 0, s>>>(g, h, base_ok, max_iter, out_counts, err_handback);
}

// ---------------------------------------------------- single-block base case

// Once the live components and edges of a Borůvka call fit in one block's
// shared memory, the remaining rounds run in one launch of the tile kernel on
// a single tile with no cut limit (every component hooks along its minimum
// edge), instead of a few launches and a host readback per round.  The live
// components get local indices 0..k-1 (their position in the active list).
__global__ void base_map_kernel(const uint32_t *act, uint32_t n_act, uint32_t *loc, u64 *offsets, uint64_t m) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_act) loc[act[i]] = i;
  if (i == 0) {
    offsets[0] = 0;
    offsets[1] = m;
  }
}

// Local ends of each list edge through the current roots (parent[] after the
// last jump points every listed end at its root, which is in the active list).
__global__ void base_pack_kernel(const uint32_t *u, const uint32_t *v, uint64_t m, const uint32_t *parent,
                                 const uint32_t *loc, uint32_t *ends) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
    ends[e] = loc[parent[u[e]]] | (loc[parent[v[e]]] << 16);
}

// New roots back to global ids: a live root takes the global id of its local
// root; vertices that were already merged keep their parent.
__global__ void base_unmap_kernel(const uint32_t *act, uint32_t n_act, const uint32_t *plocal, uint32_t *parent) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_act) return;
  const uint32_t g = act[i];
  if (parent[g] == g) parent[g] = act[plocal[i]];
}

bool launch_base_case(const uint32_t *act, uint32_t n_act, EdgeList cur, uint64_t m, uint32_t *parent, uint32_t *bits,
                      const BaseScratch &b, uint32_t *err, cudaStream_t s, int filter_heavy, u64 *wsum) {
  if (n_act == 0 || n_act > BASE_MAX_N || m > BASE_MAX_M || !cur.id) return false;
  base_map_kernel<<<(n_act + 255) / 256, 256, 0, s>>>(act, n_act, b.loc, b.offsets, m);
  if (m) base_pack_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(cur.u, cur.v, m, parent, b.loc, b.ends);
  cudaMemsetAsync(b.cutmin, 0xff, (size_t)n_act * 8, s);
  cudaMemsetAsync(b.rest_fill, 0, sizeof(u64), s);
  if (!launch_tile_contract(n_act, n_act, m, b.cutmin, b.offsets, b.ends, cur.w, cur.id, b.plocal, bits, b.rest,
                            b.rest_fill, err, s, filter_heavy, wsum))
    return false;
  base_unmap_kernel<<<(n_act + 255) / 256, 256, 0, s>>>(act, n_act, b.plocal, parent);
  return true;
}

// Fraction estimate for the automatic switch: counts how many of `samples`
// random edges (splitmix64) are local.
__global__ void tile_sample_kernel(EdgeList in, uint64_t m, uint32_t n, uint32_t B, u64 state, uint32_t samples,
                                   uint32_t *local_count) {
  uint32_t c = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < samples; i += gridDim.x * blockDim.x) {
    const uint64_t j = __umul64hi(splitmix64_at(state, i), m);
    const uint32_t u = __ldg(in.u + j), v = __ldg(in.v + j);
    c += (u < n && v < n && u != v && u / B == v / B) ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(local_count, c);
}

// ------------------------------------------------- largest component marks

// Finds the component that most endpoints of a random edge sample belong to:
// 1024 edges of the list are drawn with splitmix64, the root P[u] of each
// sample's first endpoint is taken (P fully contracted), and the most frequent
// root is written to *out (a sort in shared memory, then the longest run).
constexpr int MODE_SAMPLES = (int)GIANT_SAMPLES;
__global__ void __launch_bounds__(MODE_SAMPLES) giant_root_kernel(EdgeList in, uint64_t m_bound, const u64 *m_dev,
                                                                  u64 state, const uint32_t *P, uint32_t n,
                                                                  uint32_t *out, uint32_t *count_out) {
  const uint64_t m = m_dev ? min((uint64_t)*m_dev, m_bound) : m_bound;
  __shared__ uint32_t s_r[MODE_SAMPLES];
  __shared__ uint32_t s_best[MODE_SAMPLES / 32], s_bestv[MODE_SAMPLES / 32];
  const uint32_t t = threadIdx.x;
  uint32_t r = 0xffffffffu;
  if (m) {
    const uint32_t u = __ldg(in.u + __umul64hi(splitmix64_at(state, t), m));
    if (u < n) {  // the label of u: P may still hold chains (a bounded walk, inside 0..n-1;
                  // one cut short only picks a non-root, which marks no vertex)
      r = __ldcg(P + u);
      for (uint32_t k = 0; k < JUMP_STEPS && r < n; ++k) {
        const uint32_t q = __ldcg(P + r);
        if (q == r) break;
        r = q;
      }
    }
  }
  s_r[t] = r;
  __syncthreads();
  for (uint32_t k = 2; k <= MODE_SAMPLES; k <<= 1) {  // bitonic sort, ascending
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint32_t p = t ^ j;
      if (p > t) {
        const uint32_t a = s_r[t], b = s_r[p];
        const bool up = (t & k) == 0;
        if ((a > b) == up) {
          s_r[t] = b;
          s_r[p] = a;
        }
      }
      __syncthreads();
    }
  }
  // run length at each run start (upper bound by binary search)
  const uint32_t v = s_r[t];
  uint32_t len = 0;
  if (t == 0 || s_r[t - 1] != v) {
    uint32_t lo = t, hi = MODE_SAMPLES;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_r[mid] <= v)
        lo = mid + 1;
      else
        hi = mid;
    }
    len = lo - t;
  }
  uint32_t bl = len, bv = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t ol = __shfl_xor_sync(0xffffffffu, bl, o), ov = __shfl_xor_sync(0xffffffffu, bv, o);
    if (ol > bl || (ol == bl && ov < bv)) {
      bl = ol;
      bv = ov;
    }
  }
  if ((t & 31) == 0) {
    s_best[t >> 5] = bl;
    s_bestv[t >> 5] = bv;
  }
  __syncthreads();
  if (t == 0) {
    uint32_t l = 0, r = 0;
    for (int i = 0; i < MODE_SAMPLES / 32; ++i)
      if (s_best[i] > l || (s_best[i] == l && s_bestv[i] < r)) {
        l = s_best[i];
        r = s_bestv[i];
      }
    *out = r;
    if (count_out) *count_out = r < n ? l : 0u;  // sampled ends in that component
  }
}

// bits[v/32] bit v%32 = (P[v] == *root), for all n vertices.
__global__ void giant_bits_kernel(const uint32_t *P, uint32_t n, const uint32_t *root, uint32_t *bits) {
  const uint32_t r = *root;
  const uint64_t nw = ((uint64_t)n + 31) / 32;
  for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < nw * 32; i += (uint64_t)gridDim.x * BLOCK) {
    const bool in = i < n && __ldg(P + i) == r;
    const uint32_t word = __ballot_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0) bits[i >> 5] = word;
  }
}

// ---------------------------------------------------------------- finalize

// Output (Section 2.2; edge ids, Section 6.2): set bits of the chosen-edge
// bitmap become ascending ids; their weights are summed into a uint64.
__global__ void __launch_bounds__(BLOCK) finalize_kernel(const uint32_t *bits, uint64_t nwords, const uint32_t *w,
                                                         uint32_t *out_ids, uint32_t *out_count, u64 *total_weight,
                                                         ScanState st) {
  __shared__ uint32_t s_warp[BLOCK / 32 + 1];
  __shared__ u64 s_sum[BLOCK / 32];
  __shared__ LookbackShared s_lb;
  TileInfo t;
  if (!acquire_tile(st, nwords, t)) {
    if (t.ntiles == 0 && t.tile == 0 && threadIdx.x == 0) *out_count = 0;
    return;
  }
  const uint64_t tb = (uint64_t)t.tile * TILE;
  uint32_t wd[ITEMS], c0 = 0, c1 = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint64_t j = tb + item_off(k);
    wd[k] = j < nwords ? bits[j] : 0u;
    if (k < 4)
      c0 += __popc(wd[k]);
    else
      c1 += __popc(wd[k]);
  }
  uint32_t excl, totp;
  uint64_t obase;
  if (!tile_offsets(st, t, c0 | (c1 << 16), excl, totp, obase, s_warp, s_lb)) return;
  const uint32_t total = (totp & 0xffffu) + (totp >> 16);
  u64 wsum = 0;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint64_t pos = obase + (half == 0 ? (excl & 0xffffu) : (totp & 0xffffu) + (excl >> 16));
#pragma unroll
    for (int k = half * 4; k < half * 4 + 4; ++k) {
      uint32_t word = wd[k];
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        const uint32_t id = (uint32_t)((tb + item_off(k)) * 32 + b);
        out_ids[pos++] = id;
        if (w) wsum += __ldg(w + id);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 s = 0;
    for (int i = 0; i < BLOCK / 32; ++i) s += s_sum[i];
    if (s && w) atomicAdd(total_weight, s);
    if (t.tile == t.ntiles - 1) *out_count = (uint32_t)(obase + total);
  }
}

// *total = the sum of the WSUM_SLOTS counters (one block of WSUM_SLOTS threads).
__global__ void wsum_total_kernel(const u64 *wsum, u64 *total) {
  __shared__ u64 s_part[WSUM_SLOTS / 32];
  u64 v = wsum[threadIdx.x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int i = 0; i < WSUM_SLOTS / 32; ++i) t += s_part[i];
    *total = t;
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

// One compaction launch in tile shape (B, I): the persistent TMA kernel for
// long lists whose tiles fit two shared-memory stages, else one block per tile.
template <int MODE, int B, int I>
static void launch_compact_shaped(const CompactArgs &a, uint64_t max_count, bool aligned, cudaStream_t s) {
  constexpr int T = B * I;
  constexpr size_t stage_bytes = 16 * (size_t)T;  // compact_kernel's staging buffer
  constexpr bool tma_fits = tma_smem_bytes<B, I>() <= 200 * 1024;
  // Set once per process (a function-local static is initialised exactly once,
  // even when several host threads launch at the same time): prefer shared
  // memory over L1, allow the staging buffer, size the persistent grid.
  static const int tma_blocks = []() -> int {
    cudaFuncSetAttribute(compact_kernel<MODE, true, B, I>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(compact_kernel<MODE, true, B, I>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stage_bytes);
    int blocks = 0;
    if constexpr (tma_fits) {
      cudaFuncSetAttribute(compact_tma_kernel<MODE, B, I>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tma_smem_bytes<B, I>());
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compact_tma_kernel<MODE, B, I>, B,
                                                    tma_smem_bytes<B, I>());
      blocks = sms * per_sm;
    }
    cudaGetLastError();
    return blocks;
  }();
  const uint64_t tiles = (max_count + T - 1) / T;
  if (tiles == 0) return;
  if constexpr (tma_fits) {
    if (aligned && tma_blocks > 0 && tiles >= (uint64_t)tma_blocks * TMA_STAGES) {
      compact_tma_kernel<MODE, B, I><<<(unsigned)tma_blocks, B, tma_smem_bytes<B, I>(), s>>>(a);
      return;
    }
  }
  if (aligned) {
    compact_kernel<MODE, true, B, I><<<(unsigned)tiles, B, stage_bytes, s>>>(a);
  } else {  // unaligned lists: scalar loads in the default shape
    static const bool carveout_set = [] {  // once per process, as above
      cudaFuncSetAttribute(compact_kernel<MODE, false, BLOCK, ITEMS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
      cudaGetLastError();
      return true;
    }();
    (void)carveout_set;
    compact_kernel<MODE, false, BLOCK, ITEMS><<<(unsigned)((max_count + TILE - 1) / TILE), BLOCK, 16 * TILE, s>>>(a);
  }
}

// The warp-streamed pass over a list, if the device runs it (false: not
// launched, the caller uses the block kernels).
template <int MODE, class WS>
static bool launch_warp_stream(const CompactArgs &a, uint64_t max_count, cudaStream_t s) {
  // resident blocks of the pass (0: not available); set once per process
  static const int blocks = []() -> int {
    int dev = 0, sms = 0, per_sm = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(stream_warp_kernel<MODE, WS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)WS::smem) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_warp_kernel<MODE, WS>, WS::threads, WS::smem) ==
            cudaSuccess)
      b = sms * per_sm;
    cudaGetLastError();
    return b;
  }();
  if (blocks <= 0) return false;
  const uint64_t wtiles = (max_count + WS::tile - 1) / WS::tile;
  const uint64_t want = (wtiles + WS::warps - 1) / WS::warps;
  const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)blocks);
  stream_warp_kernel<MODE, WS><<<grid, WS::threads, WS::smem, s>>>(a);
  return true;
}

template <int MODE>
static void launch_compact_mode(const CompactArgs &a, uint64_t max_count, cudaStream_t s) {
  if (max_count == 0) return;
  const bool aligned = aligned16(a.in.u) && aligned16(a.in.v) && aligned16(a.in.w) && (!a.in.id || aligned16(a.in.id));
  if constexpr (MODE == CM_FILTER || MODE == CM_HEAVY) {
    if (aligned && launch_warp_stream<MODE, FilterWarp>(a, max_count, s)) return;
  }
  if constexpr (MODE == CM_PARTITION) {  // small light shares in the default tile shape: the warp-streamed pass
    if (aligned && a.shape == 0 && a.warp_partition && launch_warp_stream<MODE, PartitionWarp>(a, max_count, s))
      return;
  }
  if constexpr (MODE == CM_RELABEL || MODE == CM_PARTITION) {
    switch (a.shape) {  // the shapes of shape_index
      case 1: launch_compact_shaped<MODE, 128, 4>(a, max_count, aligned, s); return;
      case 2: launch_compact_shaped<MODE, 128, 8>(a, max_count, aligned, s); return;
      case 3: launch_compact_shaped<MODE, 128, 16>(a, max_count, aligned, s); return;
      case 4: launch_compact_shaped<MODE, 256, 4>(a, max_count, aligned, s); return;
      case 6: launch_compact_shaped<MODE, 256, 16>(a, max_count, aligned, s); return;
      case 7: launch_compact_shaped<MODE, 512, 4>(a, max_count, aligned, s); return;
      case 8: launch_compact_shaped<MODE, 512, 8>(a, max_count, aligned, s); return;
      case 9: launch_compact_shaped<MODE, 512, 16>(a, max_count, aligned, s); return;
      default: break;  // 0 and 5: 256 x 8
    }
  }
  launch_compact_shaped<MODE, BLOCK, ITEMS>(a, max_count, aligned, s);
}

void launch_compact(CompactMode mode, const CompactArgs &a, uint64_t max_count, cudaStream_t s) {
  switch (mode) {
    case CM_RELABEL: launch_compact_mode<CM_RELABEL>(a, max_count, s); break;
    case CM_PARTITION: launch_compact_mode<CM_PARTITION>(a, max_count, s); break;
    case CM_FILTER: launch_compact_mode<CM_FILTER>(a, max_count, s); break;
    case CM_DEDUPE: launch_compact_mode<CM_DEDUPE>(a, max_count, s); break;
    case CM_HEAVY: launch_compact_mode<CM_HEAVY>(a, max_count, s); break;
  }
}

void launch_min_edges(EdgeList in, uint64_t m, uint32_t n, int validate, KeyLayout kl, u64 *best, uint32_t *err,
                      int sms, cudaStream_t s) {
  if (m == 0) return;
  const unsigned grid = grid_for((m + (uint64_t)TILE - 1) / TILE, sms, 8);
  if (aligned16(in.u) && aligned16(in.v) && aligned16(in.w) && (!in.id || aligned16(in.id)))
    min_edges_kernel<true><<<grid, BLOCK, 0, s>>>(in, m, n, validate, kl, best, err);
  else
    min_edges_kernel<false><<<grid, BLOCK, 0, s>>>(in, m, n, validate, kl, best, err);
}

void launch_max_weight(const uint32_t *w, uint64_t m, uint32_t *out, int sms, cudaStream_t s) {
  if (m == 0) return;
  max_weight_kernel<<<grid_for((m / 4 + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(w, m, out);
}

template <int B, int I>
static void launch_hook_shaped(const HookArgs &a, uint64_t max_cand, cudaStream_t s) {
  constexpr int T = B * I;
  // a count known on the host gets one block per tile; a count in device
  // memory (up to max_cand) gets a bounded grid that strides over the tiles
  const uint64_t tiles = (max_cand + T - 1) / T;
  const unsigned grid = (unsigned)(a.ncand_dev ? std::min<uint64_t>(tiles, 152u * 8u * 256u / B) : tiles);
  // the packed layout needs no parent-chain walks: its own instantiation
  // keeps far fewer registers live (higher occupancy)
  if (a.cand)
    a.kl.packed ? hook_kernel<false, true, B, I><<<grid, B, 0, s>>>(a)
                : hook_kernel<false, false, B, I><<<grid, B, 0, s>>>(a);
  else
    a.kl.packed ? hook_kernel<true, true, B, I><<<grid, B, 0, s>>>(a)
                : hook_kernel<true, false, B, I><<<grid, B, 0, s>>>(a);
}

void launch_hook(const HookArgs &a, uint64_t max_cand, cudaStream_t s) {
  if (max_cand == 0) return;
  switch (a.shape) {  // the shapes of shape_index
    case 1: launch_hook_shaped<128, 4>(a, max_cand, s); return;
    case 2: launch_hook_shaped<128, 8>(a, max_cand, s); return;
    case 3: launch_hook_shaped<128, 16>(a, max_cand, s); return;
    case 4: launch_hook_shaped<256, 4>(a, max_cand, s); return;
    case 6: launch_hook_shaped<256, 16>(a, max_cand, s); return;
    case 7: launch_hook_shaped<512, 4>(a, max_cand, s); return;
    case 8: launch_hook_shaped<512, 8>(a, max_cand, s); return;
    case 9: launch_hook_shaped<512, 16>(a, max_cand, s); return;
    default: launch_hook_shaped<BLOCK, ITEMS>(a, max_cand, s); return;  // 0 and 5: 256 x 8
  }
}

void launch_jump(const uint32_t *act, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                 uint32_t *parent, u64 *best, int reset_best, uint32_t *flag, int sms, cudaStream_t s,
                 uint32_t max_steps, const uint32_t *groot, uint32_t *gbits) {
  if (max_count == 0) return;
  if (!act && !count_dev) {  // every vertex 0..count_host-1
    const unsigned g = grid_for(((count_host + 3) / 4 + BLOCK - 1) / BLOCK, sms, 8);
    jump_all_kernel<<<g, BLOCK, 0, s>>>(parent, best, reset_best, count_host, flag, max_steps ? max_steps : JUMP_STEPS,
                                        groot, gbits);
    return;
  }
  const unsigned grid = grid_for((max_count + JUMP_TILE - 1) / JUMP_TILE, sms, 8);
  jump_kernel<<<grid, BLOCK, 0, s>>>(act, count_dev, count_host, parent, best, reset_best, flag,
                                     max_steps ? max_steps : JUMP_STEPS);
}

void launch_range_check(const uint32_t *x, uint64_t count, uint32_t bound, uint32_t *err, int sms, cudaStream_t s) {
  if (count == 0) return;
  range_check_kernel<<<grid_for((count + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(x, count, bound, err);
}

void launch_hash_insert(EdgeList in, uint64_t m, HashSlot *table, uint64_t tmask, uint32_t *err, int sms,
                        cudaStream_t s) {
  if (m == 0) return;
  hash_insert_kernel<<<grid_for((m + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(in, m, table, tmask, err);
}

static inline uint32_t select_rank(uint32_t sample, uint32_t rank) { return rank < sample ? rank : sample / 2; }

void launch_pivot(EdgeList in, uint64_t m, const u64 *m_dev, u64 state, uint32_t sample, u64 *sample_buf,
                  u64 *pivot_out, cudaStream_t s, uint32_t rank) {
  const unsigned g = (sample + BLOCK - 1) / BLOCK;
  pivot_sample_kernel<<<g > 0 ? g : 1, BLOCK, 0, s>>>(in, m, m_dev, state, sample, sample_buf);
  pivot_select_kernel<<<1, SEL_THREADS, 0, s>>>(sample_buf, sample, select_rank(sample, rank), pivot_out);
}

size_t pivot_scratch_bytes() { return sizeof(PivotScratch); }

bool launch_pivot_coop(EdgeList in, uint64_t m, u64 state, uint32_t sample, u64 *keys, void *scratch,
                       u64 *pivot_out, cudaStream_t s, const u64 *m_dev, uint32_t rank) {
  PivotScratch *ps = static_cast<PivotScratch *>(scratch);
  uint32_t r = select_rank(sample, rank);
  void *args[] = {&in, &m, &m_dev, &state, &sample, &r, &keys, &ps, &pivot_out};
  if (cudaLaunchCooperativeKernel((const void *)pivot_coop_kernel, dim3(PSEL_BLOCKS), dim3(PSEL_THREADS), args, 0, s) ==
      cudaSuccess)
    return true;
  cudaGetLastError();
  return false;
}

void launch_wsum_total(const u64 *wsum, u64 *total, cudaStream_t s) {
  wsum_total_kernel<<<1, WSUM_SLOTS, 0, s>>>(wsum, total);
}

void launch_finalize(const uint32_t *bits, uint64_t m, const uint32_t *w, uint32_t *out_ids, uint32_t *out_count,
                     u64 *total_weight, ScanState st, cudaStream_t s) {
  const uint64_t nwords = (m + 31) / 32;
  const unsigned grid = (unsigned)(max_scan_tiles(nwords) > 0 ? max_scan_tiles(nwords) : 1);
  finalize_kernel<<<grid, BLOCK, 0, s>>>(bits, nwords, w, out_ids, out_count, total_weight, st);
}

void launch_giant_root(EdgeList in, uint64_t m, u64 state, const uint32_t *P, uint32_t n, uint32_t *root_tmp,
                       cudaStream_t s, const u64 *m_dev, uint32_t *count_out) {
  giant_root_kernel<<<1, MODE_SAMPLES, 0, s>>>(in, m, m_dev, state, P, n, root_tmp, count_out);
}

void launch_giant_bits(EdgeList in, uint64_t m, u64 state, const uint32_t *P, uint32_t n, uint32_t *root_tmp,
                       uint32_t *bits, int sms, cudaStream_t s) {
  giant_root_kernel<<<1, MODE_SAMPLES, 0, s>>>(in, m, nullptr, state, P, n, root_tmp, nullptr);
  const uint64_t threads = ((uint64_t)n + 31) / 32 * 32;
  giant_bits_kernel<<<grid_for((threads + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(P, n, root_tmp, bits);
}

void launch_tile_count(EdgeList in, uint64_t m, uint32_t n, uint32_t B, u64 *cutmin, uint32_t *count,
                       u64 *local_total, uint32_t *max_w, uint32_t *err, int sms, cudaStream_t s) {
  if (m == 0) return;
  tile_count_kernel<<<grid_for((m + TILE - 1) / TILE, sms, 8), BLOCK, 0, s>>>(in, m, n, B, cutmin, count,
                                                                              local_total, max_w, err);
}

void launch_tile_scan(const uint32_t *count, uint32_t ntiles, u64 *offsets, cudaStream_t s) {
  tile_scan_kernel<<<1, 1024, 0, s>>>(count, ntiles, offsets);
}

void launch_tile_scatter(EdgeList in, uint64_t m, uint32_t n, uint32_t B, const u64 *offsets, uint32_t *fill,
                         uint32_t *b_ends, uint32_t *b_w, uint32_t *b_id, EdgeOut cut, u64 *cut_fill, int sms,
                         cudaStream_t s) {
  if (m == 0) return;
  tile_scatter_kernel<<<grid_for((m + TILE - 1) / TILE, sms, 8), BLOCK, 0, s>>>(in, m, n, B, offsets, fill, b_ends,
                                                                                b_w, b_id, cut, cut_fill);
}

bool launch_tile_contract(uint32_t n, uint32_t B, uint64_t nlocal, const u64 *cutmin, const u64 *offsets,
                          const uint32_t *b_ends, const uint32_t *b_w, const uint32_t *b_id, uint32_t *parent,
                          uint32_t *bits, EdgeOut rest, u64 *rest_fill, uint32_t *err, cudaStream_t s,
                          int filter_heavy, u64 *wsum) {
  // set once per process, and only published once the attribute is in place
  // (another host thread must not launch with the larger size before it is)
  static const int smem_full = []() -> int {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int bytes = optin - 2048;  // static shared memory and slack
    cudaFuncSetAttribute(tile_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaGetLastError();
    return bytes;
  }();
  const size_t vbytes = (size_t)B * (8 + 8 + 4 + 4 + 4);
  if ((size_t)smem_full <= vbytes) return false;
  const uint32_t ntiles = (uint32_t)(((uint64_t)n + B - 1) / B);
  // Edge capacity: a quarter above the mean bucket (so more tiles share an
  // SM), at most what the in-place compaction holds and the block can get.
  // Larger buckets run from global memory.
  uint64_t want = nlocal / ntiles;
  want = ((want + want / 4 + 256) + 31) / 32 * 32;
  uint64_t cap = min(want, (uint64_t)TC_EPT * TC_THREADS);
  cap = min(cap, ((size_t)smem_full - vbytes) / 12);
  const size_t bytes = vbytes + (size_t)cap * 12;
  tile_contract_kernel<<<ntiles, TC_THREADS, bytes, s>>>(n, B, cutmin, offsets, b_ends, b_w, b_id, (uint32_t)cap,
                                                         parent, bits, rest, rest_fill, err, filter_heavy, wsum);
  return true;
}

void launch_tile_sample(EdgeList in, uint64_t m, uint32_t n, uint32_t B, u64 state, uint32_t samples,
                        uint32_t *local_count, cudaStream_t s) {
  if (m == 0) return;
  tile_sample_kernel<<<(samples + 255) / 256, 256, 0, s>>>(in, m, n, B, state, samples, local_count);
}

void launch_iota(uint32_t *p, uint64_t n, int sms, cudaStream_t s) {
  if (n == 0) return;
  iota_kernel<<<grid_for((n + BLOCK - 1) / BLOCK, sms, 8), BLOCK, 0, s>>>(p, n);
}


}  // namespace mstgpu
