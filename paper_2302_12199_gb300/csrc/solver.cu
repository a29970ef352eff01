// Host side of libmstgpu: the C ABI declared in include/mst.h, the Borůvka
// round loop (Section 2.3, Alg. 1), the Filter-Borůvka recursion (Alg. 2), the
// batched disjoint-union solve and the step entry points.
//
// Device memory: each handle owns a CUDA memory pool; every solve allocates its
// scratch from it in stream order and returns it at the end, so repeated solves
// reuse the same memory without device-wide synchronisation.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"
#include "mst.h"

using namespace mstgpu;

struct mst_ctx {
  int device = 0;
  mst_config cfg;
  mst_status last = MST_OK;
  int last_cuda = 0;         // cudaError_t behind the last MST_ERR_CUDA
  int last_cuda_line = 0;    // source line of the call that returned it
  int sms = 152;
  cudaMemPool_t pool = nullptr;
  DevState *ds = nullptr;    // device
  DevState *hs = nullptr;    // page-locked, mapped host mirror of ds, written by readback_kernel
  DevState *hs_dev = nullptr;   // its device-side address
  uint32_t *hflag = nullptr;    // mapped host word: sequence number of the last completed readback
  uint32_t *hflag_dev = nullptr;
  uint32_t rb_seq = 0;
  uint64_t readbacks = 0;
  u64 *hres = nullptr;       // pinned host words for the forest size and weight of the host entry points
  u64 *status = nullptr;     // scan status words
  uint64_t status_cap = 0;   // in tiles
  uint32_t epoch = 0;
  u64 *sample_buf = nullptr;
  uint32_t sample_cap = 0;
  void *pivot_scratch = nullptr;  // histograms of the multi-block pivot selection
  u64 *wsum = nullptr;            // WSUM_SLOTS counters of the chosen weights (zeroed per solve)
  uint64_t pivot_counter = 0;
  uint64_t solves = 0, planned = 0;
  uint64_t plan_fallbacks = 0;  // planned Filter-Borůvka solves that started over on the host-driven path
  // per-kernel-class event timing (mst_profile_enable)
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes, min_bytes;  // fixed parts known at launch (see prof_end)
    int slot[3];              // counts the launch's bytes scale with (-1: none)
    double per[3], per_min[3];
  };
  bool prof_on = false;
  uint32_t prof_mask = ~0u;  // classes that get event timing (the others: launches and bytes only)
  cudaStream_t cap_stream = nullptr;  // stream the round graphs are captured on
  cudaStream_t copy_stream = nullptr; // input copies of mst_solve_host_many
  cudaEvent_t in_ready[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr};
  // device buffers of the host entry points (inputs, two sets; the forest),
  // grown on demand and kept: outside the pool, so that the solves' scratch
  // never splits them and the pool never has to grow while a copy runs
  void *hin[2] = {nullptr, nullptr};
  size_t hin_cap[2] = {0, 0};
  void *hout = nullptr;
  size_t hout_cap = 0;
  // the two ping-pong edge lists of the Borůvka rounds (u, v, w, id each),
  // kept by the handle and grown on demand: with stable addresses and a stable
  // capacity bound, one captured round graph serves every Borůvka call (and
  // every later solve) of the handle
  void *rl_mem = nullptr;
  uint64_t rl_cap = 0;  // edges per list
  GraphRounds *grounds = nullptr;     // device state of the graph round loop
  struct RoundGraph {
    u64 sig;  // every pointer and size the graph was built with
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  };
  std::vector<RoundGraph> round_graphs;  // most recently used first
  std::vector<u64> round_sigs_seen;      // shapes met once (a graph is built on the second meeting)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> prof_pending;
  mst_kernel_stats prof[MST_K_COUNT];
};

namespace {

constexpr int TILE_ITEMS = 2048;

// The CUDA error of the call that made the current API call fail (per host
// thread; record() moves it into the handle).
thread_local int tl_cuda_error = 0;
thread_local int tl_cuda_line = 0;

#define CK(call)                                \
  do {                                          \
    const cudaError_t _e = (call);              \
    if (_e != cudaSuccess) {                    \
      tl_cuda_error = (int)_e;                  \
      tl_cuda_line = __LINE__;                  \
      return MST_ERR_CUDA;                      \
    }                                           \
  } while (0)

#define TRY(expr)                     \
  do {                                \
    mst_status _st = (expr);          \
    if (_st != MST_OK) return _st;    \
  } while (0)

u64 host_mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
u64 host_splitmix64_at(u64 s, u64 i) { return host_mix64(s + (i + 1ULL) * 0x9e3779b97f4a7c15ULL); }

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int ceil_log2(uint64_t x) {
  int l = 0;
  while ((1ULL << l) < x) ++l;
  return l;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// A stream-ordered device allocation from the handle's pool.
struct Buf {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  Buf() = default;
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  ~Buf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  mst_status alloc(mst_ctx *c, size_t bytes, cudaStream_t st) {
    release();
    s = st;
    if (bytes == 0) bytes = 256;
    if (cudaMallocFromPoolAsync(&p, bytes, c->pool, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return MST_ERR_OOM;
    }
    return MST_OK;
  }
  template <class T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

// An edge list buffer: four uint32 arrays of `cap` entries in one allocation.
struct ListBuf {
  Buf mem;
  uint64_t cap = 0;
  EdgeOut out{};
  mst_status alloc(mst_ctx *c, uint64_t n_edges, cudaStream_t s) {
    const uint64_t stride = round_up(n_edges * 4 + 16, 256);
    TRY(mem.alloc(c, stride * 4, s));
    char *b = mem.as<char>();
    out = EdgeOut{(uint32_t *)b, (uint32_t *)(b + stride), (uint32_t *)(b + 2 * stride), (uint32_t *)(b + 3 * stride)};
    cap = n_edges;
    return MST_OK;
  }
  EdgeList list() const { return EdgeList{out.u, out.v, out.w, out.id}; }
};

// A view of one of the handle's round lists.
struct RoundList {
  EdgeOut out{};
  uint64_t cap = 0;
  EdgeList list() const { return EdgeList{out.u, out.v, out.w, out.id}; }
};

// Points X and Y at the handle's round lists, first growing them (a quarter
// above `need`, in steps of 2^16 edges) when they hold fewer than `need`
// edges.  The growth is stream-ordered on s: the old lists are freed after the
// work queued on s so far (calls return only after their work is done, so no
// earlier call still reads them), and nothing waits for the whole device, which
// other threads may be using (or capturing graphs on) at the same time.
mst_status round_lists(mst_ctx *c, uint64_t need, RoundList &X, RoundList &Y, cudaStream_t s) {
  if (!c->rl_mem || c->rl_cap < need) {
    const uint64_t want = round_up(std::max<uint64_t>(need + need / 4, 1ULL << 16), 1ULL << 16);
    if (c->rl_mem) CK(cudaFreeAsync(c->rl_mem, s));
    c->rl_mem = nullptr;
    c->rl_cap = 0;
    if (cudaMallocAsync(&c->rl_mem, 8 * round_up(want * 4 + 16, 256), s) != cudaSuccess) {
      cudaGetLastError();
      c->rl_mem = nullptr;
      return MST_ERR_OOM;
    }
    c->rl_cap = want;
  }
  const uint64_t stride = round_up(c->rl_cap * 4 + 16, 256);
  char *b = static_cast<char *>(c->rl_mem);
  RoundList *L[2] = {&X, &Y};
  for (int k = 0; k < 2; ++k) {
    char *q = b + (size_t)4 * k * stride;
    L[k]->out = EdgeOut{(uint32_t *)q, (uint32_t *)(q + stride), (uint32_t *)(q + 2 * stride), (uint32_t *)(q + 3 * stride)};
    L[k]->cap = c->rl_cap;
  }
  return MST_OK;
}

mst_status ensure_status(mst_ctx *c, uint64_t max_items, cudaStream_t s) {
  const uint64_t tiles = (max_items + TILE_ITEMS - 1) / TILE_ITEMS + 1;
  if (tiles <= c->status_cap) return MST_OK;
  // stream-ordered, like the round lists: no wait for the whole device
  if (c->status) CK(cudaFreeAsync(c->status, s));
  c->status = nullptr;
  c->status_cap = 0;
  const uint64_t cap = next_pow2(tiles < 4096 ? 4096 : tiles);
  if (cudaMallocAsync(&c->status, cap * sizeof(u64), s) != cudaSuccess) {
    cudaGetLastError();
    c->status = nullptr;
    return MST_ERR_OOM;
  }
  CK(cudaMemsetAsync(c->status, 0, cap * sizeof(u64), s));
  c->status_cap = cap;
  c->epoch = 0;
  CK(cudaMemsetAsync(c->ds->tile_ctr, 0, sizeof(c->ds->tile_ctr), s));
  return MST_OK;
}

ScanState next_scan(mst_ctx *c, int total_slot) {
  if (++c->epoch >= (1u << 30)) {  // epochs wrapped: clear the status words (practically never)
    cudaDeviceSynchronize();
    cudaMemset(c->status, 0, c->status_cap * sizeof(u64));
    cudaMemset(c->ds->tile_ctr, 0, sizeof(c->ds->tile_ctr));
    c->epoch = 1;
  }
  return ScanState{c->status, c->ds->tile_ctr, c->epoch, &c->ds->count[total_slot], &c->ds->err, c->cfg.spin_limit};
}

cudaEvent_t take_event(mst_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Opens a record around the next launch(es) of class `kind` on `s`; -1 when
// profiling is off.  Only the classes in prof_mask are timed with events.
int prof_begin(mst_ctx *c, cudaStream_t s, int kind) {
  if (!c->prof_on) return -1;
  mst_ctx::ProfRec r{};
  if (c->prof_mask >> kind & 1u) {
    r.a = take_event(c);
    r.b = take_event(c);
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
  }
  c->prof_pending.push_back(r);
  return (int)c->prof_pending.size() - 1;
}

// Closes a record: `bytes` known at launch, plus count[slot] * per for counts the
// kernel itself produces (read at the next readback).  `min_bytes` (< 0: the
// same as `bytes`) replaces the fixed part in the method's own count, for a
// pass that reads more than the method needs (the filter re-reads the light
// edges of its list along with the heavy ones).
void prof_end(mst_ctx *c, cudaStream_t s, int idx, int kind, double bytes, int slot1 = -1, double per1 = 0,
              int slot2 = -1, double per2 = 0, double min_bytes = -1.0) {
  if (idx < 0) return;
  mst_ctx::ProfRec &r = c->prof_pending[idx];
  if (r.b) cudaEventRecord(r.b, s);
  r.kind = kind;
  r.bytes = bytes;
  r.min_bytes = min_bytes < 0.0 ? bytes : min_bytes;
  r.slot[0] = slot1;
  r.per[0] = r.per_min[0] = per1;
  r.slot[1] = slot2;
  r.per[1] = r.per_min[1] = per2;
  r.slot[2] = -1;
  r.per[2] = r.per_min[2] = 0.0;
}

// Byte terms of a launch whose list lengths are device counts: besides the
// fixed parts, term i adds count[slot] * per to the bytes moved and
// count[slot] * per_min to the method's own count.
struct ProfTerm {
  int slot;
  double per, per_min;
};
void prof_end_terms(mst_ctx *c, cudaStream_t s, int idx, int kind, double bytes, double min_bytes, ProfTerm t0,
                    ProfTerm t1 = {-1, 0, 0}, ProfTerm t2 = {-1, 0, 0}) {
  if (idx < 0) return;
  mst_ctx::ProfRec &r = c->prof_pending[idx];
  if (r.b) cudaEventRecord(r.b, s);
  r.kind = kind;
  r.bytes = bytes;
  r.min_bytes = min_bytes;
  const ProfTerm t[3] = {t0, t1, t2};
  for (int i = 0; i < 3; ++i) {
    r.slot[i] = t[i].slot;
    r.per[i] = t[i].per;
    r.per_min[i] = t[i].per_min;
  }
}

// After a stream synchronisation: folds the finished records into the totals.
void prof_resolve(mst_ctx *c) {
  for (auto &r : c->prof_pending) {
    float ms = 0.f;
    if (r.b) cudaEventSynchronize(r.b);  // done on the device; let the runtime see it
    if (r.a && cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    mst_kernel_stats &k = c->prof[r.kind];
    k.launches += 1;
    k.ms += ms;
    double b = 0.0, bm = 0.0;
    for (int i = 0; i < 3; ++i)
      if (r.slot[i] >= 0) {
        b += (double)c->hs->count[r.slot[i]] * r.per[i];
        bm += (double)c->hs->count[r.slot[i]] * r.per_min[i];
      }
    k.bytes += r.bytes + b;
    k.min_bytes += r.min_bytes + bm;
    if (r.a) {
      c->ev_pool.push_back(r.a);
      c->ev_pool.push_back(r.b);
    }
  }
  c->prof_pending.clear();
}

#define PROF(kind, bytes, slot1, per1, slot2, per2, launch)       \
  do {                                                           \
    const int _p = prof_begin(c, s, kind);                       \
    launch;                                                      \
    prof_end(c, s, _p, kind, bytes, slot1, per1, slot2, per2);   \
  } while (0)

// A launch whose bytes follow device counts (see prof_end_terms; the
// trailing arguments are its ProfTerms).
#define PROF_TERMS(kind, bytes, min_bytes, launch, ...)                  \
  do {                                                                   \
    const int _p = prof_begin(c, s, kind);                               \
    launch;                                                              \
    prof_end_terms(c, s, _p, kind, bytes, min_bytes, __VA_ARGS__);       \
  } while (0)

// The same with the method's own fixed byte count `min_bytes` (see prof_end).
#define PROF_MIN(kind, bytes, min_bytes, slot1, per1, slot2, per2, launch)     \
  do {                                                                         \
    const int _p = prof_begin(c, s, kind);                                     \
    launch;                                                                    \
    prof_end(c, s, _p, kind, bytes, slot1, per1, slot2, per2, min_bytes);      \
  } while (0)

// Copies the device state into the mapped host mirror, then publishes `seq`
// in the mapped flag word (one warp, after everything before it on the
// stream).  The system-scope fence orders the mirror's words before the flag.
__global__ void readback_kernel(const DevState *ds, DevState *hs, uint32_t *flag, uint32_t seq) {
  constexpr int words = (int)(sizeof(DevState) / 4);
  const uint32_t *src = reinterpret_cast<const uint32_t *>(ds);
  volatile uint32_t *dst = reinterpret_cast<volatile uint32_t *>(hs);
  for (int i = threadIdx.x; i < words; i += 32) dst[i] = src[i];
  __threadfence_system();
  __syncwarp();
  if (threadIdx.x == 0) *reinterpret_cast<volatile uint32_t *>(flag) = seq;
}

// The host side of a readback: the state of the device counters and flags
// after all work queued on s so far.  The host spins on the mapped flag
// (a few microseconds after the GPU gets there, where a copy plus a stream
// synchronisation costs about ten); after about a second without the flag it
// falls back to synchronising the stream, which also reports a CUDA error.
// Error bits in `tolerated` are left for the caller to act on.
mst_status readback(mst_ctx *c, cudaStream_t s, uint32_t tolerated = 0) {
  static_assert(sizeof(DevState) % 4 == 0, "DevState is copied in words");
  const uint32_t seq = ++c->rb_seq;
  ++c->readbacks;
  readback_kernel<<<1, 32, 0, s>>>(c->ds, c->hs_dev, c->hflag_dev, seq);
  CK(cudaGetLastError());
  bool seen = false;
  for (uint64_t spin = 0; spin < (1ULL << 26); ++spin) {
    if (__atomic_load_n(c->hflag, __ATOMIC_ACQUIRE) == seq) {
      seen = true;
      break;
    }
    if ((spin & 0x3ffff) == 0x3ffff && cudaStreamQuery(s) != cudaErrorNotReady) {  // a fault: stop waiting
      seen = __atomic_load_n(c->hflag, __ATOMIC_ACQUIRE) == seq;
      break;
    }
  }
  if (!seen) CK(cudaStreamSynchronize(s));
  if (__atomic_load_n(c->hflag, __ATOMIC_ACQUIRE) != seq) return MST_ERR_CUDA;
  prof_resolve(c);
  const uint32_t err = c->hs->err & ~tolerated;
  if (err & ERR_VERTEX) return MST_ERR_VERTEX_RANGE;
  if (err & ERR_TABLE) return MST_ERR_INVALID_ARG;
  if (err) return MST_ERR_INTERNAL;
  return MST_OK;
}

// Clears the error word, the jump flag and both tile counters (err, jump_flag
// and tile_ctr are adjacent in DevState).  Called at the start of every solve
// and step call, so that a launch that failed earlier cannot leave a counter
// behind for the scans of this call.
mst_status clear_device_flags(mst_ctx *c, cudaStream_t s) {
  static_assert(offsetof(DevState, tile_ctr) == 2 * sizeof(uint32_t), "DevState layout");
  CK(cudaMemsetAsync(c->ds, 0, 4 * sizeof(uint32_t), s));
  return MST_OK;
}

bool aligned4(const void *p) { return ((uintptr_t)p & 3u) == 0; }

// Zeroes the counters that the unordered compactions of one step add into
// (edges, active vertices, the dedupe temporary).
mst_status zero_counters(mst_ctx *c, cudaStream_t s) {
  static_assert(CNT_EDGES == 0 && CNT_ACTIVE == 1 && CNT_TMP == 2, "counter layout");
  CK(cudaMemsetAsync(&c->ds->count[0], 0, 3 * sizeof(u64), s));
  return MST_OK;
}

// The same plus the jump flag (one memset over jump_flag .. count[2]; the
// error word stays): a Borůvka round's first operation, so that the round's
// jump launch needs no memset of its own.
mst_status zero_round_state(mst_ctx *c, cudaStream_t s) {
  static_assert(offsetof(DevState, jump_flag) == sizeof(uint32_t) && offsetof(DevState, count) == 4 * sizeof(uint32_t),
                "DevState layout");
  CK(cudaMemsetAsync(&c->ds->jump_flag, 0, offsetof(DevState, count) + 3 * sizeof(u64) - offsetof(DevState, jump_flag),
                     s));
  return MST_OK;
}

// Per-solve state: vertex arrays and the chosen-edge bitmap.
struct Solve {
  mst_ctx *c;
  cudaStream_t s;
  uint32_t n;
  uint64_t m;
  Buf best_b, parent_b, act_b[2], bits_b;
  const uint32_t *src = nullptr, *dst = nullptr;  // input endpoints, indexed by edge id
  const uint32_t *w_in = nullptr;                 // input weights
  KeyLayout kl{0, 0, 0};  // unpacked unless choose_layout() packs
  bool layout_set = false;
  // unpacked keys: ends of each edge by id as written with the current list
  Buf cur_b;
  uint32_t *cur_u = nullptr, *cur_v = nullptr;
  mst_status cur_alloc() {
    if (kl.packed || cur_u) return MST_OK;
    const uint64_t stride = round_up(m * 4 + 16, 256);
    TRY(cur_b.alloc(c, stride * 2, s));
    cur_u = cur_b.as<uint32_t>();
    cur_v = (uint32_t *)((char *)cur_b.p + stride);
    return MST_OK;
  }
  // Sets the recording of ends by id on a pass that writes a list (unpacked keys).
  void record_ends(CompactArgs &a) const {
    a.cur_u = (layout_set && !kl.packed) ? cur_u : nullptr;
    a.cur_v = (layout_set && !kl.packed) ? cur_v : nullptr;
  }
  u64 *best = nullptr;
  uint32_t *parent = nullptr, *act[2] = {nullptr, nullptr}, *bits = nullptr;
  int wbits = 32;  // bits of the largest weight (set with the key layout)
  int rounds = 0;
  int shape = 0;   // tile shape of the partition / filter compactions and the hook (shape_index)
  int rshape = 1;  // tile shape of the relabel compaction (relabel_shape_index)

  Solve(mst_ctx *c_, cudaStream_t s_, uint32_t n_, uint64_t m_)
      : c(c_), s(s_), n(n_), m(m_), shape(shape_index(c_->cfg.block_threads, c_->cfg.items_per_thread)),
        rshape(relabel_shape_index(c_->cfg.relabel_block_threads, c_->cfg.relabel_items_per_thread)) {}

  mst_status init(uint32_t *parent_external = nullptr, uint32_t *bits_external = nullptr) {
    TRY(best_b.alloc(c, (size_t)n * 8, s));
    best = best_b.as<u64>();
    CK(cudaMemsetAsync(best, 0xff, (size_t)n * 8, s));
    if (parent_external) {
      parent = parent_external;
    } else {
      TRY(parent_b.alloc(c, (size_t)n * 4, s));
      parent = parent_b.as<uint32_t>();
    }
    launch_iota(parent, n, c->sms, s);
    for (int i = 0; i < 2; ++i) {
      TRY(act_b[i].alloc(c, (size_t)n * 4, s));
      act[i] = act_b[i].as<uint32_t>();
    }
    if (bits_external) {
      bits = bits_external;
    } else {
      const size_t words = (m + 31) / 32;
      TRY(bits_b.alloc(c, words * 4, s));
      bits = bits_b.as<uint32_t>();
      CK(cudaMemsetAsync(bits, 0, words * 4, s));
    }
    TRY(ensure_status(c, (uint64_t)n > m ? (uint64_t)n : m, s));
    TRY(clear_device_flags(c, s));
    CK(cudaMemsetAsync(c->wsum, 0, WSUM_SLOTS * sizeof(u64), s));
    return MST_OK;
  }

  // Picks the relaxation key layout (KeyLayout): the far end of the edge goes
  // into the key when the largest weight, the edge ids and the vertex ids fit
  // into 63 bits together (the top bit stays clear, so no key equals INF).
  mst_status choose_layout(const uint32_t *w) {
    CK(cudaMemsetAsync(&c->ds->max_w, 0, sizeof(uint32_t), s));
    launch_max_weight(w, m, &c->ds->max_w, c->sms, s);
    TRY(readback(c, s));
    set_layout();
    return cur_alloc();
  }
  // From the largest weight in hs->max_w (read back by the caller).
  void set_layout() {
    layout_set = true;
    const int vb = n > 1 ? 64 - __builtin_clzll((unsigned long long)(n - 1)) : 1;
    const int ib = m > 1 ? 64 - __builtin_clzll((unsigned long long)(m - 1)) : 1;
    const uint32_t mw = c->hs->max_w;
    const int wb = mw ? 32 - __builtin_clz(mw) : 0;
    wbits = wb;
    kl = KeyLayout{wb + ib + vb <= 63 ? 1 : 0, vb, ib};
  }

  // Pointer jumping over the listed vertices (act == nullptr: all n) until
  // every one points to its root; the first launch may reset best[].
  // One pointer-jumping launch over the list (or all n), with the flag cleared
  // first; the flag is read back by the caller's next readback.
  mst_status jump_launch(const uint32_t *act_list, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                         int reset_best, const uint32_t *groot = nullptr, uint32_t *gbits = nullptr,
                         bool flag_clear = false) {
    if (!flag_clear) CK(cudaMemsetAsync(&c->ds->jump_flag, 0, sizeof(uint32_t), s));
    const int slot = count_dev ? CNT_ACTIVE : -1;
    const double fixed = count_dev ? 0.0 : (8.0 + (gbits ? 0.125 : 0.0)) * (double)count_host;
    PROF(MST_K_JUMP, fixed, slot, reset_best ? 20.0 : 12.0, -1, 0.0,
         launch_jump(act_list, count_dev, count_host, max_count, parent, best, reset_best, &c->ds->jump_flag,
                     c->sms, s, c->cfg.jump_steps, groot, gbits));
    return MST_OK;
  }

  // Relaunches (after a readback) while the flag says a walk fell short.
  mst_status jump_finish(const uint32_t *act_list, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                         const uint32_t *groot = nullptr, uint32_t *gbits = nullptr) {
    for (int it = 0; c->hs->jump_flag; ++it) {
      if (it > 64) return MST_ERR_INTERNAL;
      TRY(jump_launch(act_list, count_dev, count_host, max_count, 0, groot, gbits));
      TRY(readback(c, s));
    }
    return MST_OK;
  }

  // flag_clear: the jump flag is known to be zero (zero_round_state began the
  // round and nothing since touched it)
  mst_status jump_until_stars(const uint32_t *act_list, const u64 *count_dev, uint64_t count_host, uint64_t max_count,
                              int reset_best, const uint32_t *groot = nullptr, uint32_t *gbits = nullptr,
                              bool flag_clear = false) {
    TRY(jump_launch(act_list, count_dev, count_host, max_count, reset_best, groot, gbits, flag_clear));
    TRY(readback(c, s));
    return jump_finish(act_list, count_dev, count_host, max_count, groot, gbits);
  }

  // Parallel-edge removal is optional (Section 2.3).  `auto` keeps parallel
  // edges: on GNM, RGG and RMAT inputs the two extra passes and the table cost
  // more than the parallel edges they remove save in later rounds.
  bool want_dedupe(int round, uint64_t cur_m) const {
    (void)round;
    return (c->cfg.dedupe == MST_DEDUPE_HASH || c->cfg.dedupe == MST_DEDUPE_SORT) && cur_m > 0;
  }

  // Borůvka rounds (Section 2.3) on the list E of mE edges whose endpoints are
  // current component roots; merged roots get their new root in parent[].
  // best_ready: best[] already holds this list's minEdges (relaxed by the pass
  // that wrote the list).
  // ends_rec: cur_u/cur_v hold E's ends by id (written with E); otherwise the
  // hook of the first round walks from the input ends.
  mst_status boruvka(EdgeList E, uint64_t mE, bool validate, bool best_ready = false, bool ends_rec = false) {
    if (mE == 0) return MST_OK;
    if (!layout_set) TRY(choose_layout(w_in ? w_in : E.w));
    // round 0: minEdges straight from the stored list (atomic minima, or
    // segmented minima over the ends sorted by vertex), then hook and jump
    if (!best_ready) {
      bool done_sorted = false;
      if (c->cfg.min_edges_sort && 2 * mE < (1ULL << 32)) {
        Buf me_b;
        TRY(me_b.alloc(c, min_edges_sort_scratch_bytes(mE, c->sms), s));
        const double passes = (double)((ceil_log2((uint64_t)n + 1) + 7) / 8);
        PROF(MST_K_MIN_EDGES, (12.0 + 24.0 + 2.0 * (32.0 * passes + 20.0)) * (double)mE, -1, 0.0, -1, 0.0,
             done_sorted = launch_min_edges_sort(E, mE, n, validate ? 1 : 0, kl, best, &c->ds->err, me_b.p, c->sms,
                                                 s));
      }
      if (!done_sorted)
        PROF(MST_K_MIN_EDGES, 12.0 * (double)mE, -1, 0.0, -1, 0.0,
             launch_min_edges(E, mE, n, validate ? 1 : 0, kl, best, &c->ds->err, c->sms, s));
    }
    TRY(zero_round_state(c, s));
    HookArgs ha{};
    ha.shape = shape;
    ha.cand = nullptr;
    ha.ncand = n;
    ha.best = best;
    ha.kl = kl;
    const bool rec = ends_rec && cur_u;  // ends recorded with the list, or walk from the input
    ha.src = rec ? cur_u : src;
    ha.dst = rec ? cur_v : dst;
    ha.parent = parent;
    ha.chosen_bits = bits;
    ha.active_out = act[0];
    ha.counter = &c->ds->count[CNT_ACTIVE];
    ha.err = &c->ds->err;
    ha.wsum = c->wsum;
    PROF(MST_K_HOOK, 8.0 * (double)n, CNT_ACTIVE, 8.0, -1, 0.0, launch_hook(ha, n, s));
    TRY(jump_until_stars(act[0], &c->ds->count[CNT_ACTIVE], 0, n, 1, nullptr, nullptr, true));
    uint64_t n_act = c->hs->count[CNT_ACTIVE];
    ++rounds;

    RoundList X, Y;  // the handle's round lists (lists only shrink within a call: mE edges suffice)
    TRY(round_lists(c, mE, X, Y, s));
    ListBuf T;
    Buf table_b;
    EdgeList cur = E;
    uint64_t cur_m = mE;
    int a = 0;
    const int bound = 2 * (ceil_log2(n) + 2);
    for (int r = 1; n_act > 0; ++r) {
      if (r > bound) return MST_ERR_INTERNAL;
      if (base_case_fits(cur, cur_m, n_act)) return base_case(cur, cur_m, act[a], (uint32_t)n_act);
      if (c->cfg.graph_rounds && cur.u == X.out.u && cur.id && !want_dedupe(r, cur_m)) {
        bool used = false, done = false;
        int ran = 0;
        TRY(graph_rounds(X, Y, cur, cur_m, n_act, a, bound - r, used, done, ran));
        if (used) {
          r += ran;
          rounds += ran;
          if (done || n_act == 0 || cur_m == 0) return MST_OK;
          --r;  // the loop's ++r
          continue;
        }
      }
      RoundList &out = (cur.u == X.out.u) ? Y : X;
      TRY(zero_round_state(c, s));
      CompactArgs ca{};
      ca.shape = rshape;
      ca.in = cur;
      ca.m = cur_m;
      ca.out = out.out;
      ca.label = parent;
      ca.n = n;
      ca.kl = kl;
      const double in_bytes = (cur.id ? 16.0 : 12.0) * (double)cur_m;
      if (!want_dedupe(r, cur_m)) {
        ca.best = best;
        record_ends(ca);
        ca.st = next_scan(c, CNT_EDGES);
        PROF(MST_K_RELABEL_MIN, in_bytes, CNT_EDGES, 16.0, -1, 0.0, launch_compact(CM_RELABEL, ca, cur_m, s));
      } else if (c->cfg.dedupe == MST_DEDUPE_SORT) {
        // relabel into T, then keep each pair's lightest edge by sorting
        // (Section 2.3 parallel-edge removal, sort variant) and relax best[]
        if (T.cap < cur_m) TRY(T.alloc(c, cur_m, s));
        ca.out = T.out;
        ca.st = next_scan(c, CNT_TMP);
        PROF(MST_K_DEDUPE, in_bytes, CNT_TMP, 16.0, -1, 0.0, launch_compact(CM_RELABEL, ca, cur_m, s));
        TRY(readback(c, s));
        const uint64_t mT = c->hs->count[CNT_TMP];
        Buf sd_b;
        TRY(sd_b.alloc(c, sort_dedupe_scratch_bytes(mT, c->sms), s));
        CompactArgs cd{};
        cd.shape = shape;
        cd.in = T.list();
        cd.m = mT;
        cd.out = out.out;
        cd.best = best;
        cd.kl = kl;
        record_ends(cd);
        cd.n = n;
        cd.st = next_scan(c, CNT_EDGES);
        const int passes = (wbits + kl.idbits + 7) / 8 + (2 * kl.vbits + 7) / 8;
        PROF(MST_K_DEDUPE, (32.0 * passes + 56.0) * (double)mT, CNT_EDGES, 16.0, -1, 0.0,
             launch_sort_dedupe(T.list(), mT, kl.vbits, wbits, kl.idbits, cd, sd_b.p, c->sms, s));
      } else {
        // relabel into T while inserting every pair into the hash table, then
        // keep each pair's minimum (Section 2.3 parallel-edge removal; the
        // hash variant of Section 6.2) and relax best[] with the final slots
        if (T.cap < cur_m) TRY(T.alloc(c, cur_m, s));
        const uint64_t slots = next_pow2(2 * cur_m < 1024 ? 1024 : 2 * cur_m);
        TRY(table_b.alloc(c, slots * sizeof(HashSlot), s));
        CK(cudaMemsetAsync(table_b.p, 0xff, slots * sizeof(HashSlot), s));
        ca.out = T.out;
        ca.table = table_b.as<HashSlot>();
        ca.tmask = slots - 1;
        ca.hash_insert = 1;
        ca.st = next_scan(c, CNT_TMP);
        PROF(MST_K_DEDUPE, in_bytes, CNT_TMP, 16.0, -1, 0.0, launch_compact(CM_RELABEL, ca, cur_m, s));
        CompactArgs cd{};
        cd.shape = shape;
        cd.in = T.list();
        cd.m = cur_m;
        cd.m_dev = &c->ds->count[CNT_TMP];
        cd.out = out.out;
        cd.table = ca.table;
        cd.tmask = ca.tmask;
        cd.best = best;
        cd.kl = kl;
        record_ends(cd);
        cd.n = n;
        cd.st = next_scan(c, CNT_EDGES);
        PROF(MST_K_DEDUPE, 0.0, CNT_TMP, 16.0, CNT_EDGES, 16.0, launch_compact(CM_DEDUPE, cd, cur_m, s));
      }
      HookArgs hb{};
      hb.shape = shape;
      hb.cand = act[a];
      hb.ncand = n_act;
      hb.best = best;
      hb.kl = kl;
      hb.src = cur_u ? cur_u : src;
      hb.dst = cur_v ? cur_v : dst;
      hb.parent = parent;
      hb.chosen_bits = bits;
      hb.active_out = act[1 - a];
      hb.counter = &c->ds->count[CNT_ACTIVE];
      hb.err = &c->ds->err;
      hb.wsum = c->wsum;
      PROF(MST_K_HOOK, 12.0 * (double)n_act, CNT_ACTIVE, 8.0, -1, 0.0, launch_hook(hb, n_act, s));
      TRY(jump_until_stars(act[1 - a], &c->ds->count[CNT_ACTIVE], 0, n_act, 1, nullptr, nullptr, true));
      table_b.release();
      a = 1 - a;
      n_act = c->hs->count[CNT_ACTIVE];
      cur = out.list();
      cur_m = c->hs->count[CNT_EDGES];
      ++rounds;
      if (cur_m == 0) break;
    }
    return MST_OK;
  }

  // The round graph over lists X, Y and active lists A (see build_round_graph),
  // from the handle's cache.  Not cached yet: built at once when `always`,
  // else only when the same shape is asked for again (a graph pays for its
  // capture and instantiation only when its shape comes back); exec stays
  // null when it is not built.  err_handback: the device-driven mode's error
  // word (see launch_round_pre), or null.
  mst_status round_graph(RoundList &X, RoundList &Y, uint32_t *const A[2], uint32_t max_iter, uint32_t *err_handback,
                         bool always, cudaGraphExec_t &exec) {
    exec = nullptr;
    // launch bounds baked into the graph: the lists' capacity and n (the
    // kernels read the actual counts from device memory), so the graph does
    // not depend on this call's sizes
    const uint64_t cap = std::min(X.cap, Y.cap), nmax = n;
    if (!c->grounds) CK(cudaMalloc(&c->grounds, sizeof(GraphRounds)));
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int base_ok = (c->cfg.base_case && !err_handback) ? 1 : 0;
    const int jl = c->cfg.graph_jump_launches;
    const RoundList *L[2] = {&X, &Y};
    // A built graph is reused when every value baked into it is unchanged.
    u64 sig = 0x2302121990ULL;
    auto fold = [&](u64 v) { sig = host_mix64(sig ^ (v + 0x9e3779b97f4a7c15ULL)); };
    for (int i = 0; i < 2; ++i) {
      fold((u64)L[i]->out.u), fold((u64)L[i]->out.v), fold((u64)L[i]->out.w), fold((u64)L[i]->out.id);
      fold((u64)A[i]);
    }
    const u64 vals[] = {(u64)parent,  (u64)best,    (u64)bits,     (u64)cur_u,  (u64)cur_v,
                        (u64)src,     (u64)dst,     (u64)c->status, (u64)c->ds,  (u64)c->grounds,
                        (u64)kl.packed, (u64)kl.vbits, (u64)kl.idbits, (u64)n,     (u64)cap,
                        (u64)nmax,    (u64)jl,      (u64)base_ok,  (u64)max_iter, (u64)c->sms,
                        (u64)shape,   (u64)err_handback};
    for (u64 v : vals) fold(v);
    for (size_t i = 0; i < c->round_graphs.size(); ++i)
      if (c->round_graphs[i].sig == sig) {
        const mst_ctx::RoundGraph hit = c->round_graphs[i];
        c->round_graphs.erase(c->round_graphs.begin() + i);
        c->round_graphs.insert(c->round_graphs.begin(), hit);
        exec = hit.exec;
        return MST_OK;
      }
    if (!always) {
      auto &seen = c->round_sigs_seen;
      const bool again = std::find(seen.begin(), seen.end(), sig) != seen.end();
      if (!again) {
        seen.insert(seen.begin(), sig);
        if (seen.size() > 64) seen.pop_back();
        return MST_OK;
      }
    }
    return build_round_graph(sig, L, A, cap, nmax, base_ok, jl, max_iter, err_handback, exec);
  }

  // Rounds of a Borůvka call as one CUDA graph launch (the round loop without
  // host round trips): a conditional WHILE node repeats a body of two rounds
  // (list X -> Y, then Y -> X; the active lists alternate the same way) while
  // the device sees active vertices and edges.  It hands the state back to the
  // host when the base case fits, when a round's pointer jumping needs more
  // than the four launches a round holds, or at the round bound.  Counts live
  // in device memory; nothing in the body waits for the host.
  mst_status graph_rounds(RoundList &X, RoundList &Y, EdgeList &cur, uint64_t &cur_m, uint64_t &n_act, int &a,
                          int rounds_left, bool &used, bool &done, int &ran) {
    used = false;
    done = false;
    ran = 0;
    const uint32_t max_iter = (uint32_t)(rounds_left > 2 ? rounds_left / 2 : 1);
    uint32_t *A[2] = {act[a], act[1 - a]};
    cudaGraphExec_t exec = nullptr;
    TRY(round_graph(X, Y, A, max_iter, nullptr, false, exec));
    if (!exec) return MST_OK;  // the first time, the host runs the rounds
    GraphRounds *g = c->grounds;
    used = true;
    launch_round_init(g, cur_m, n_act, s);
    PROF(MST_K_GRAPH, 0.0, -1, 0.0, -1, 0.0, CK(cudaGraphLaunch(exec, s)));
    TRY(readback(c, s));
    const u64 info = c->hs->count[CNT_TMP];
    const uint32_t reason = (uint32_t)(info & 0xff), slot = (uint32_t)((info >> 8) & 0xff);
    ran = 2 * (int)(info >> 16);
    if (reason == ROUNDS_BOUND || reason == ROUNDS_RUNNING || slot > 1) return MST_ERR_INTERNAL;
    cur_m = c->hs->count[CNT_EDGES];
    n_act = c->hs->count[CNT_ACTIVE];
    cur = (slot == 0 ? X : Y).list();
    if (slot == 1) a = 1 - a;
    if (reason == ROUNDS_DONE) {
      done = true;
      return MST_OK;
    }
    if (reason == ROUNDS_JUMP) TRY(jump_until_stars(act[a], nullptr, n_act, n_act, 0));
    return MST_OK;
  }

  // Captures and instantiates the round graph: an entry kernel that decides
  // whether the loop runs at all, then a conditional WHILE node whose body is
  // two rounds (slot 0 -> 1, slot 1 -> 0), each compaction (relabel + minEdges
  // relaxation), hooking, `jl` pointer-jumping launches and a check; the body
  // ends with the kernel that sets the loop condition.
  mst_status build_round_graph(u64 sig, const RoundList *const L[2], uint32_t *const A[2], uint64_t cap, uint64_t nmax,
                               int base_ok, int jl, uint32_t max_iter, uint32_t *err_handback,
                               cudaGraphExec_t &exec_out) {
    GraphRounds *g = c->grounds;
    cudaStream_t cs = c->cap_stream;
    struct Owned {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaStream_t capturing = nullptr;
      ~Owned() {
        if (capturing) {  // an error during capture: end it so the stream is usable again
          cudaGraph_t dummy = nullptr;
          cudaStreamEndCapture(capturing, &dummy);
          cudaGetLastError();
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
      }
    } o;
    CK(cudaGraphCreate(&o.graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, o.graph, 0, cudaGraphCondAssignDefault));
    // entry: the kernel that decides whether the loop runs at all
    CK(cudaStreamBeginCaptureToGraph(cs, o.graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    o.capturing = cs;
    launch_round_pre(g, h, &c->ds->count[CNT_EDGES], err_handback, cs);
    {
      cudaGraph_t captured = nullptr;
      o.capturing = nullptr;
      CK(cudaStreamEndCapture(cs, &captured));
    }
    cudaGraphNode_t pre = nullptr;
    size_t nodes = 1;
    CK(cudaGraphGetNodes(o.graph, &pre, &nodes));
    if (nodes != 1 || !pre) return MST_ERR_INTERNAL;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, o.graph, &pre, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    o.capturing = cs;
    for (int half = 0; half < 2; ++half) {
      const int in = half, out = 1 - half;
      CompactArgs ca{};
      ca.shape = rshape;
      ca.in = L[in]->list();
      ca.m = cap;
      ca.m_dev = &g->ce[in];
      ca.out = L[out]->out;
      ca.label = parent;
      ca.n = n;
      ca.kl = kl;
      ca.best = best;
      record_ends(ca);
      ca.st = ScanState{c->status, c->ds->tile_ctr, 0, &g->ce[out], &c->ds->err, c->cfg.spin_limit};
      launch_compact(CM_RELABEL, ca, cap, cs);
      HookArgs hb{};
      hb.shape = shape;
      hb.cand = A[in];
      hb.ncand_dev = &g->ca[in];
      hb.best = best;
      hb.kl = kl;
      hb.src = cur_u ? cur_u : src;
      hb.dst = cur_v ? cur_v : dst;
      hb.parent = parent;
      hb.chosen_bits = bits;
      hb.active_out = A[out];
      hb.counter = &g->ca[out];
      hb.err = &c->ds->err;
      hb.wsum = c->wsum;
      launch_hook(hb, nmax, cs);
      // pointer jumping: jl launches of up to 256 steps each; only the last
      // launch reports a vertex short of its root
      for (int k = 0; k < jl; ++k)
        launch_jump(A[out], &g->ca[out], 0, nmax, parent, best, k == 0 ? 1 : 0, k == jl - 1 ? &g->jflag : &g->jdummy,
                    c->sms, cs, 256);
      if (half == 0) launch_round_check(g, base_ok, err_handback, cs);
    }
    launch_round_cond(g, h, base_ok, max_iter, &c->ds->count[CNT_EDGES], err_handback, cs);
    cudaGraph_t captured = nullptr;
    o.capturing = nullptr;
    CK(cudaStreamEndCapture(cs, &captured));
    CK(cudaGraphInstantiate(&o.exec, o.graph, 0));
    c->round_graphs.insert(c->round_graphs.begin(), mst_ctx::RoundGraph{sig, o.graph, o.exec});
    exec_out = o.exec;
    o.graph = nullptr;
    o.exec = nullptr;
    while (c->round_graphs.size() > 16) {
      cudaGraphExecDestroy(c->round_graphs.back().exec);
      cudaGraphDestroy(c->round_graphs.back().graph);
      c->round_graphs.pop_back();
    }
    return MST_OK;
  }

  // The last rounds of a Borůvka call in one block once the live components
  // and edges fit in its shared memory (the list must carry ids).
  bool base_case_fits(EdgeList cur, uint64_t cur_m, uint64_t n_act) const {
    return c->cfg.base_case && cur.id && n_act > 0 && n_act <= BASE_MAX_N && cur_m <= BASE_MAX_M;
  }
  mst_status base_case(EdgeList cur, uint64_t cur_m, const uint32_t *act_list, uint32_t n_act) {
    const size_t a_loc = round_up((size_t)n * 4 + 4, 256), a_ends = round_up(BASE_MAX_M * 4, 256);
    const size_t a_cut = (size_t)BASE_MAX_N * 8, a_off = 256, a_pl = (size_t)BASE_MAX_N * 4;
    Buf sb;
    TRY(sb.alloc(c, a_loc + a_ends + a_cut + a_off + a_pl + 4 * a_ends + 256, s));
    char *p = sb.as<char>();
    BaseScratch b{};
    b.loc = (uint32_t *)p;
    p += a_loc;
    b.ends = (uint32_t *)p;
    p += a_ends;
    b.cutmin = (u64 *)p;
    p += a_cut;
    b.offsets = (u64 *)p;
    p += a_off;
    b.plocal = (uint32_t *)p;
    p += a_pl;
    b.rest = EdgeOut{(uint32_t *)p, (uint32_t *)(p + a_ends), (uint32_t *)(p + 2 * a_ends), (uint32_t *)(p + 3 * a_ends)};
    p += 4 * a_ends;
    b.rest_fill = (u64 *)p;
    bool launched = false;
    PROF(MST_K_BASE, 16.0 * (double)cur_m + 28.0 * (double)n_act, -1, 0.0, -1, 0.0,
         launched = launch_base_case(act_list, n_act, cur, cur_m, parent, bits, b, &c->ds->err, s, c->cfg.tile_filter,
                                     c->wsum));
    if (!launched) return MST_ERR_INTERNAL;
    // no readback: the base case produces no count the host needs, and an
    // error bit it sets stays latched until the next readback reports it
    return MST_OK;
  }

  // Local preprocessing (Section 4.1) on vertex-range tiles.  When applied,
  // parent[] holds every vertex's tile root, the contracted edges are marked,
  // and the input relabelled by those roots (internal edges dropped) is left in
  // `out` (fused with the first minEdges when relax is set).  `auto` (-1)
  // applies it only if at least 10% of the edges are local (Section 6.2),
  // estimated from a sample first.
  mst_status tile_preprocess(const uint32_t *w, bool relax, ListBuf &out, uint64_t &m_out, bool &applied) {
    applied = false;
    const uint32_t B = c->cfg.tile_vertices;
    const EdgeList in{src, dst, w, nullptr};
    if (c->cfg.tile_contract == 0 || m == 0) return MST_OK;
    if (c->cfg.tile_contract < 0) {
      CK(cudaMemsetAsync(&c->ds->local_samples, 0, sizeof(uint32_t), s));
      launch_tile_sample(in, m, n, B, 0x51ced0ULL, 4096, &c->ds->local_samples, s);
      TRY(readback(c, s));
      if (c->hs->local_samples < 410) return MST_OK;  // < 10% of 4096 samples local
    }
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + B - 1) / B);
    Buf cut_b, cnt_b, off_b, fill_b, bucket_b;
    TRY(cut_b.alloc(c, (size_t)n * 8, s));
    TRY(cnt_b.alloc(c, (size_t)ntiles * 4, s));
    TRY(off_b.alloc(c, ((size_t)ntiles + 1) * 8, s));
    TRY(fill_b.alloc(c, (size_t)ntiles * 4, s));
    CK(cudaMemsetAsync(cut_b.p, 0xff, (size_t)n * 8, s));
    CK(cudaMemsetAsync(cnt_b.p, 0, (size_t)ntiles * 4, s));
    CK(cudaMemsetAsync(fill_b.p, 0, (size_t)ntiles * 4, s));
    CK(cudaMemsetAsync(&c->ds->count[CNT_AUX], 0, sizeof(u64), s));
    CK(cudaMemsetAsync(&c->ds->max_w, 0, sizeof(uint32_t), s));
    PROF(MST_K_TILE, 12.0 * (double)m + 8.0 * (double)n, -1, 0.0, -1, 0.0,
         launch_tile_count(in, m, n, B, cut_b.as<u64>(), cnt_b.as<uint32_t>(), &c->ds->count[CNT_AUX],
                           &c->ds->max_w, &c->ds->err, c->sms, s));
    TRY(readback(c, s));
    if (!layout_set) set_layout();
    TRY(cur_alloc());
    const uint64_t nlocal = c->hs->count[CNT_AUX];
    if (c->cfg.tile_contract < 0 && nlocal * 10 < m) return MST_OK;
    PROF(MST_K_TILE, 12.0 * (double)ntiles, -1, 0.0, -1, 0.0, launch_tile_scan(cnt_b.as<uint32_t>(), ntiles, off_b.as<u64>(), s));
    const uint64_t stride = round_up(nlocal * 4 + 16, 256);
    TRY(bucket_b.alloc(c, stride * 3, s));
    char *bb = bucket_b.as<char>();
    // the cut edges (written by the scatter) and the local edges that remain
    // between tile components (appended by the contraction)
    const uint64_t mcut = m;
    ListBuf cutl;
    TRY(cutl.alloc(c, mcut, s));
    CK(cudaMemsetAsync(&c->ds->count[CNT_CUT], 0, sizeof(u64), s));
    PROF(MST_K_TILE, 12.0 * (double)m + 12.0 * (double)nlocal + 16.0 * (double)(m - nlocal), -1, 0.0, -1, 0.0,
         launch_tile_scatter(in, m, n, B, off_b.as<u64>(), fill_b.as<uint32_t>(), (uint32_t *)bb,
                             (uint32_t *)(bb + stride), (uint32_t *)(bb + 2 * stride), cutl.out,
                             &c->ds->count[CNT_CUT], c->sms, s));
    bool launched = false;
    PROF(MST_K_TILE, 12.0 * (double)nlocal + 12.0 * (double)n, -1, 0.0, -1, 0.0,
         launched = launch_tile_contract(n, B, nlocal, cut_b.as<u64>(), off_b.as<u64>(), (uint32_t *)bb,
                                         (uint32_t *)(bb + stride), (uint32_t *)(bb + 2 * stride), parent, bits,
                                         cutl.out, &c->ds->count[CNT_CUT], &c->ds->err, s, c->cfg.tile_filter,
                                         c->wsum));
    if (!launched) return MST_ERR_INVALID_ARG;  // tile too large for shared memory
    // the cut edges, relabelled to the tile roots, are the contracted graph
    TRY(out.alloc(c, mcut, s));
    TRY(zero_counters(c, s));
    CompactArgs ca{};
    ca.shape = rshape;
    ca.in = cutl.list();
    ca.m = mcut;
    ca.m_dev = &c->ds->count[CNT_CUT];
    ca.out = out.out;
    ca.label = parent;
    ca.n = n;
    ca.kl = kl;
    ca.best = relax ? best : nullptr;
    record_ends(ca);
    ca.st = next_scan(c, CNT_EDGES);
    PROF(MST_K_RELABEL_MIN, 0.0, CNT_CUT, 16.0, CNT_EDGES, 16.0, launch_compact(CM_RELABEL, ca, mcut, s));
    TRY(readback(c, s));
    m_out = c->hs->count[CNT_EDGES];
    applied = true;
    return MST_OK;
  }

  // Rank of the pivot in its sample, and the expected light part of a list of
  // mE edges split there (Alg. 2 takes the sample median: rank s / 2, half).
  uint32_t pivot_rank() const {
    const uint32_t smp = c->cfg.pivot_sample;
    const uint32_t r = (uint32_t)std::floor((double)c->cfg.pivot_quantile * (double)smp);
    return r < smp ? r : smp - 1;
  }
  uint64_t light_est(uint64_t mE) const { return (uint64_t)((double)c->cfg.pivot_quantile * (double)mE); }
  // the warp-streamed partition pays off while the light share is small
  int warp_partition() const { return c->cfg.pivot_quantile <= 0.125f ? 1 : 0; }

  bool is_sparse(uint64_t mE) const {
    return mE < c->cfg.filter_min_edges || 2.0 * (double)mE <= (double)c->cfg.filter_max_avg_degree * (double)n;
  }

  // Full pointer doubling of parent[] over all n vertices (the contraction of
  // the representative array P before filtering, Section 5).
  mst_status compress_all() { return jump_until_stars(nullptr, nullptr, n, n, 0); }

  mst_status reset_best() {
    CK(cudaMemsetAsync(best, 0xff, (size_t)n * 8, s));
    return MST_OK;
  }

  // Contracts P (as compress_all) and marks the vertices of the component
  // that most sampled edges of E touch: the filter drops an edge with both
  // ends marked without reading P.  The sampled ends are walked to their roots
  // first; the marks are written by the contraction pass itself.  Only the
  // first launch is issued here: its flag is read back with the filter's
  // count, and contract_finish completes the rare contraction that needs more.
  mst_status contract_and_mark_start(EdgeList E, uint64_t mE, u64 state, Buf &bits_b) {
    TRY(bits_b.alloc(c, ((size_t)n + 31) / 32 * 4, s));
    launch_giant_root(E, mE, state, parent, n, &c->ds->giant_root, s, nullptr, &c->ds->giant_count);
    return jump_launch(nullptr, nullptr, n, n, 0, &c->ds->giant_root, bits_b.as<uint32_t>());
  }
  mst_status contract_and_mark_finish(Buf &bits_b) {
    return jump_finish(nullptr, nullptr, n, n, &c->ds->giant_root, bits_b.as<uint32_t>());
  }

  // Rec-Filter-MST (Alg. 2).  best_ready: best[] holds E's minEdges already.
  // With `carry` (levels below the top), a small set of filtered heavy edges
  // is not solved at this level but handed back in *carry (Section 6.3: small
  // filtered sets go back up and join the heavy edges one level up); the
  // caller appends it to its own filtered edges.  Filtering against a P that
  // lacks those edges' contractions only keeps more edges, never drops an MSF
  // edge.
  mst_status filter(EdgeList E, uint64_t mE, bool is_input, int depth, bool best_ready = false,
                    bool ends_rec = false, ListBuf *carry = nullptr, uint64_t *carry_m = nullptr) {
    if (carry_m) *carry_m = 0;
    if (is_sparse(mE) || depth >= 40) return boruvka(E, mE, is_input, best_ready, ends_rec);
    if (best_ready) TRY(reset_best());
    const u64 state = host_splitmix64_at(c->cfg.seed, c->pivot_counter++);
    PROF(MST_K_PIVOT, 16.0 * (double)c->cfg.pivot_sample, -1, 0.0, -1, 0.0,
         if (!launch_pivot_coop(E, mE, state, c->cfg.pivot_sample, c->sample_buf, c->pivot_scratch, &c->ds->pivot,
                                s, nullptr, pivot_rank())) launch_pivot(E, mE, nullptr, state, c->cfg.pivot_sample,
                                                                        c->sample_buf, &c->ds->pivot, s,
                                                                        pivot_rank()));
    const double in_bytes = (E.id ? 16.0 : 12.0) * (double)mE;
    // the light part goes straight to Borůvka rounds when it will be sparse:
    // the partition pass then also performs that call's first minEdges
    const bool fuse_light = is_sparse(light_est(mE));
    ListBuf L;
    TRY(L.alloc(c, mE, s));
    CompactArgs cp{};
    cp.shape = shape;
    cp.warp_partition = warp_partition();
    cp.in = E;
    cp.m = mE;
    cp.out = L.out;
    cp.pivot_dev = &c->ds->pivot;
    cp.n = n;
    cp.validate = is_input ? 1 : 0;
    if (!layout_set) {
      if (fuse_light) TRY(choose_layout(w_in));  // the pass below relaxes already
      else {
        CK(cudaMemsetAsync(&c->ds->max_w, 0, sizeof(uint32_t), s));
        cp.max_w = &c->ds->max_w;
      }
    }
    cp.best = fuse_light ? best : nullptr;
    cp.kl = kl;
    record_ends(cp);
    cp.st = next_scan(c, CNT_EDGES);
    TRY(zero_counters(c, s));
    PROF(MST_K_PARTITION, in_bytes, CNT_EDGES, 16.0, -1, 0.0, launch_compact(CM_PARTITION, cp, mE, s));
    TRY(readback(c, s));
    if (cp.max_w && is_input) {
      set_layout();
      TRY(cur_alloc());
    }
    const uint64_t mL = c->hs->count[CNT_EDGES];
    const u64 pivot = c->hs->pivot;
    if (mL == 0 || mL == mE) {  // no progress from this pivot: solve the list directly
      L.mem.release();
      if (fuse_light) TRY(reset_best());
      return boruvka(E, mE, is_input, false, ends_rec);
    }
    ListBuf lcarry;
    uint64_t lcarry_m = 0;
    const bool carrying = c->cfg.filter_carry != 0;
    TRY(filter(L.list(), mL, false, depth + 1, fuse_light, cp.cur_u != nullptr, carrying ? &lcarry : nullptr,
               carrying ? &lcarry_m : nullptr));
    L.mem.release();
    Buf giant_b;
    TRY(contract_and_mark_start(E, mE, host_mix64(state), giant_b));
    ListBuf H;
    TRY(H.alloc(c, mE - mL + lcarry_m, s));
    CompactArgs cf{};
    cf.shape = shape;
    cf.in = E;
    cf.m = mE;
    cf.out = H.out;
    cf.label = parent;
    cf.giant_bits = giant_b.as<uint32_t>();
    cf.giant_count = &c->ds->giant_count;
    cf.pivot = pivot;
    cf.n = n;
    cf.best = best;  // the survivors are expected to be sparse (Theorem 1)
    cf.kl = kl;
    record_ends(cf);
    TRY(zero_counters(c, s));
    // the method reads only the heavy edges of E (the light ones went into L)
    const double heavy_bytes = (E.id ? 16.0 : 12.0) * (double)(mE - mL);
    ListBuf C;
    // The filter runs against P before the contraction's flag is known: a P
    // that is not fully contracted (labels that are ancestors, not roots) only
    // keeps more edges, but H's ends must be roots, so in that rare case the
    // contraction is finished and the pass runs again on fresh minEdges.
    for (int attempt = 0;; ++attempt) {
      cf.st = next_scan(c, CNT_EDGES);
      if (c->cfg.filter_split) {
        // two passes: the streaming pass keeps the heavy edges not inside the
        // giant component (bitmap gathers only), the filter then gathers the
        // labels for that short list
        TRY(C.alloc(c, mE - mL, s));
        CompactArgs ch{};
        ch.shape = shape;
        ch.in = E;
        ch.m = mE;
        ch.out = C.out;
        ch.giant_bits = cf.giant_bits;
        ch.pivot = pivot;
        ch.n = n;
        ch.kl = kl;
        ch.st = next_scan(c, CNT_TMP);
        PROF_MIN(MST_K_FILTER, in_bytes, heavy_bytes, CNT_TMP, 16.0, -1, 0.0, launch_compact(CM_HEAVY, ch, mE, s));
        cf.in = C.list();
        cf.m = mE - mL;
        cf.m_dev = &c->ds->count[CNT_TMP];
        cf.giant_bits = nullptr;
        PROF(MST_K_FILTER, 0.0, CNT_TMP, 16.0, CNT_EDGES, 16.0, launch_compact(CM_FILTER, cf, mE - mL, s));
      } else {
        PROF_MIN(MST_K_FILTER, in_bytes, heavy_bytes, CNT_EDGES, 16.0, -1, 0.0,
                 launch_compact(CM_FILTER, cf, mE, s));
      }
      TRY(readback(c, s));
      if (!c->hs->jump_flag) break;
      if (attempt > 0) return MST_ERR_INTERNAL;
      TRY(contract_and_mark_finish(giant_b));
      TRY(reset_best());
      TRY(zero_counters(c, s));
      cf.in = E;
      cf.m = mE;
      cf.m_dev = nullptr;
      cf.giant_bits = giant_b.as<uint32_t>();
    }
    C.mem.release();
    giant_b.release();
    uint64_t mH = c->hs->count[CNT_EDGES];
    bool relaxed = true;  // best[] holds the minEdges of H
    if (lcarry_m) {       // the light recursion's unsolved edges join H (their ends are current roots)
      for (int k = 0; k < 4; ++k) {
        uint32_t *dstp = k == 0 ? H.out.u : k == 1 ? H.out.v : k == 2 ? H.out.w : H.out.id;
        const uint32_t *srcp = k == 0 ? lcarry.out.u : k == 1 ? lcarry.out.v : k == 2 ? lcarry.out.w : lcarry.out.id;
        CK(cudaMemcpyAsync(dstp + mH, srcp, lcarry_m * 4, cudaMemcpyDeviceToDevice, s));
      }
      mH += lcarry_m;
      TRY(reset_best());  // minEdges over the union runs again
      relaxed = false;
      lcarry.mem.release();
    }
    if (carry && mH <= n / 8) {  // small: hand it to the level above
      *carry_m = mH;
      std::swap(carry->mem.p, H.mem.p);
      std::swap(carry->mem.s, H.mem.s);
      carry->cap = H.cap;
      carry->out = H.out;
      return MST_OK;
    }
    return filter(H.list(), mH, false, depth + 1, relaxed, cf.cur_u != nullptr);
  }

  // ---------------------------------------------------------------- planned
  // Filter-Borůvka (Alg. 2) with the recursion laid out by the host ahead of
  // time and every list length kept in device memory.  The top-level
  // partition's light count (one readback, which also brings the largest
  // weight for the key layout) fixes the plan: light lists shrink by the
  // pivot's quantile q from level to level (q of each list is light: 1/2 for
  // the sample median of Alg. 2), so the host knows how many levels reach
  // isSparse and gives each list a capacity a little above q of its parent's.
  // The levels then run without the host reading anything:
  // pivot and partition from device counts, and the deepest light list and
  // each level's filtered heavy edges solved by Borůvka rounds whose first
  // hooking runs before the round graph and whose loop the device ends.  A
  // list that outgrows its capacity (ERR_OVERFLOW), a round that would need
  // the host (ERR_HANDBACK) or a contraction left short (the jump flag) makes
  // the result unusable, and the caller starts over on the host-driven path.
  // Where the estimate stops the recursion a level early or late the forest
  // is the same: isSparse only steers the work.
  bool plan_eligible() const {
    const mst_config &f = c->cfg;
    return f.filter_plan && f.graph_rounds && !f.filter_carry && !f.filter_split && !f.min_edges_sort &&
           f.dedupe != MST_DEDUPE_HASH && f.dedupe != MST_DEDUPE_SORT && !is_sparse(m);
  }
  // Capacity planned for the light list of a list of at most `cap` edges:
  // its expected light share (pivot_quantile, 1/2 for the sample median) plus
  // 1/32 of it and 2^16 (the light share of a list split at a quantile of a
  // sample of 2^16 keys strays from it by at most about 2^-9 of the list).
  uint64_t light_cap(uint64_t cap) const {
    return std::min<uint64_t>(cap, light_est(cap) + cap / 32 + (1ULL << 16));
  }
  // The round lists of a plan: the deepest light list, and each level's
  // filtered heavy edges in turn: room for n / (2q) of them with a light share
  // q (n at the median), or for every edge of the input if that is fewer.  By
  // Theorem 1 the heavy edges that survive a filter against the forest of a
  // sample of rate q number about n / q in expectation at most; on the graphs
  // measured they are far fewer.
  uint64_t plan_round_edges(uint64_t deepest_cap) const {
    const double per_n = 0.5 / (double)c->cfg.pivot_quantile;
    const uint64_t heavy = std::min<uint64_t>((uint64_t)(per_n * (double)n), m);
    return std::max<uint64_t>(std::max<uint64_t>(deepest_cap, heavy), 1ULL << 16);
  }

  // Borůvka rounds on the list in round list X whose length is count[slot]
  // (best[] holds its minEdges; ends_rec: its ends were recorded by id as it
  // was written): the first hooking over all n vertices and its pointer
  // jumping, then the round graph.
  mst_status boruvka_planned(RoundList &X, RoundList &Y, int slot, bool ends_rec, cudaGraphExec_t exec) {
    GraphRounds *g = c->grounds;
    launch_round_init_dev(g, &c->ds->count[slot], std::min(X.cap, Y.cap), s);
    HookArgs ha{};
    ha.shape = shape;
    ha.cand = nullptr;
    ha.ncand = n;
    ha.best = best;
    ha.kl = kl;
    const bool rec = ends_rec && cur_u;
    ha.src = rec ? cur_u : src;
    ha.dst = rec ? cur_v : dst;
    ha.parent = parent;
    ha.chosen_bits = bits;
    ha.active_out = act[0];
    ha.counter = &g->ca[0];
    ha.err = &c->ds->err;
    ha.wsum = c->wsum;
    PROF(MST_K_HOOK, 8.0 * (double)n, -1, 0.0, -1, 0.0, launch_hook(ha, n, s));
    const int jl = c->cfg.graph_jump_launches;
    PROF(MST_K_JUMP, 0.0, -1, 0.0, -1, 0.0,
         for (int k = 0; k < jl; ++k) launch_jump(act[0], &g->ca[0], 0, n, parent, best, k == 0 ? 1 : 0,
                                                  k == jl - 1 ? &g->jflag : &g->jdummy, c->sms, s, 256));
    PROF(MST_K_GRAPH, 0.0, -1, 0.0, -1, 0.0, CK(cudaGraphLaunch(exec, s)));
    ++rounds;
    return MST_OK;
  }

  // planned: set once the call is committed to the plan (its outcome is then
  // known after the final readback).  Unset on return: the caller runs the
  // host-driven recursion instead, after restart().
  mst_status filter_planned(bool &planned) {
    planned = false;
    const uint64_t m0 = m;
    const bool leaf_top = is_sparse(light_est(m0));  // the top level's light list is expected to be the deepest
    if (leaf_top && !layout_set) TRY(choose_layout(w_in));
    Buf piv_b, gbits_b;
    TRY(piv_b.alloc(c, LVL_MAX * sizeof(u64), s));
    TRY(gbits_b.alloc(c, ((size_t)n + 31) / 32 * 4, s));
    u64 *piv = piv_b.as<u64>();
    uint32_t *gbits = gbits_b.as<uint32_t>();
    CK(cudaMemsetAsync(&c->ds->count[CNT_LVL], 0, 2 * LVL_MAX * sizeof(u64), s));
    const uint64_t cap1 = light_cap(m0);
    RoundList X, Y;
    TRY(round_lists(c, plan_round_edges(leaf_top ? cap1 : 0), X, Y, s));
    ListBuf L1;
    if (!leaf_top) TRY(L1.alloc(c, cap1, s));

    // level 0: pivot and partition of the input (vertex ids checked here)
    const EdgeList in{src, dst, w_in, nullptr};
    u64 state[LVL_MAX];
    state[0] = host_splitmix64_at(c->cfg.seed, c->pivot_counter++);
    PROF(MST_K_PIVOT, 16.0 * (double)c->cfg.pivot_sample, -1, 0.0, -1, 0.0,
         if (!launch_pivot_coop(in, m0, state[0], c->cfg.pivot_sample, c->sample_buf, c->pivot_scratch, &piv[0], s,
                                nullptr, pivot_rank()))
             launch_pivot(in, m0, nullptr, state[0], c->cfg.pivot_sample, c->sample_buf, &piv[0], s, pivot_rank()));
    CompactArgs cp{};
    cp.shape = shape;
    cp.warp_partition = warp_partition();
    cp.in = in;
    cp.m = m0;
    cp.out = leaf_top ? X.out : L1.out;
    cp.out_cap = leaf_top ? X.cap : L1.cap;
    cp.pivot_dev = &piv[0];
    cp.n = n;
    cp.validate = 1;
    if (!layout_set) {
      CK(cudaMemsetAsync(&c->ds->max_w, 0, sizeof(uint32_t), s));
      cp.max_w = &c->ds->max_w;
    }
    cp.best = leaf_top ? best : nullptr;
    cp.kl = kl;
    record_ends(cp);
    cp.st = next_scan(c, CNT_LVL + 1);
    PROF(MST_K_PARTITION, 12.0 * (double)m0, CNT_LVL + 1, 16.0, -1, 0.0, launch_compact(CM_PARTITION, cp, m0, s));
    TRY(readback(c, s, ERR_OVERFLOW));
    if (c->hs->err & ERR_OVERFLOW) return MST_OK;  // outgrew the plan
    const uint64_t m1 = c->hs->count[CNT_LVL + 1];
    if (m1 == 0 || m1 == m0) return MST_OK;  // no progress from this pivot
    if (cp.max_w) {
      set_layout();
      TRY(cur_alloc());
    }
    // the plan: lists 1 .. K-1 are partitioned, list K is the deepest
    int K = 1;
    uint64_t caps[LVL_MAX + 1];
    caps[0] = m0;
    caps[1] = leaf_top ? X.cap : m1;
    for (uint64_t est = m1; !is_sparse(est); est = light_est(est)) {
      if (K + 1 >= LVL_MAX) return MST_OK;  // deeper than a plan holds
      caps[K + 1] = light_cap(caps[K]);
      ++K;
    }
    if (leaf_top != (K == 1)) return MST_OK;  // the light count moved the deepest level: host-driven
    const uint64_t need = plan_round_edges(caps[K]);
    if (need > X.cap) TRY(round_lists(c, need, X, Y, s));  // (not when leaf_top: X already holds list 1)
    planned = true;
    CK(cudaMemsetAsync(&c->ds->jump_flag, 0, sizeof(uint32_t), s));
    uint32_t *A[2] = {act[0], act[1]};
    cudaGraphExec_t exec = nullptr;
    TRY(round_graph(X, Y, A, (uint32_t)(ceil_log2(n) + 2), &c->ds->err, true, exec));
    if (!exec) return MST_ERR_INTERNAL;

    // light lists 2 .. K (list K into X, relaxing best[] for its first round)
    std::unique_ptr<ListBuf[]> Lb(new ListBuf[K + 1]);
    EdgeList E[LVL_MAX + 1];
    E[0] = in;
    E[1] = leaf_top ? X.list() : L1.list();
    for (int k = 1; k < K; ++k) {
      const bool last = k + 1 == K;
      if (!last) TRY(Lb[k + 1].alloc(c, caps[k + 1], s));
      state[k] = host_splitmix64_at(c->cfg.seed, c->pivot_counter++);
      const u64 *mk = &c->ds->count[CNT_LVL + k];
      PROF(MST_K_PIVOT, 16.0 * (double)c->cfg.pivot_sample, -1, 0.0, -1, 0.0,
           if (!launch_pivot_coop(E[k], caps[k], state[k], c->cfg.pivot_sample, c->sample_buf, c->pivot_scratch,
                                  &piv[k], s, mk, pivot_rank()))
               launch_pivot(E[k], caps[k], mk, state[k], c->cfg.pivot_sample, c->sample_buf, &piv[k], s,
                            pivot_rank()));
      CompactArgs pk{};
      pk.shape = shape;
      pk.warp_partition = warp_partition();
      pk.in = E[k];
      pk.m = caps[k];
      pk.m_dev = mk;
      pk.out = last ? X.out : Lb[k + 1].out;
      pk.out_cap = last ? X.cap : Lb[k + 1].cap;
      pk.pivot_dev = &piv[k];
      pk.n = n;
      pk.best = last ? best : nullptr;
      pk.kl = kl;
      record_ends(pk);
      pk.st = next_scan(c, CNT_LVL + k + 1);
      PROF_TERMS(MST_K_PARTITION, 0.0, 0.0, launch_compact(CM_PARTITION, pk, caps[k], s),
                 ProfTerm{CNT_LVL + k, 16.0, 16.0}, ProfTerm{CNT_LVL + k + 1, 16.0, 16.0});
      E[k + 1] = last ? X.list() : Lb[k + 1].list();
    }
    TRY(boruvka_planned(X, Y, CNT_LVL + K, cur_u != nullptr, exec));

    // levels K-1 .. 0: contract P and mark the giant component, filter the
    // level's heavy edges into X, and solve them
    for (int k = K - 1; k >= 0; --k) {
      if (k + 1 >= 2 && k + 1 < K) Lb[k + 1].mem.release();  // list k+1 is not read again
      const u64 *mk = k == 0 ? nullptr : &c->ds->count[CNT_LVL + k];
      launch_giant_root(E[k], caps[k], host_mix64(state[k]), parent, n, &c->ds->giant_root, s, mk,
                        &c->ds->giant_count);
      PROF(MST_K_JUMP, 8.125 * (double)n, -1, 0.0, -1, 0.0,
           launch_jump(nullptr, nullptr, n, n, parent, best, 0, &c->ds->jump_flag, c->sms, s, 4096,
                       &c->ds->giant_root, gbits));
      CompactArgs cf{};
      cf.shape = shape;
      cf.in = E[k];
      cf.m = caps[k];
      cf.m_dev = mk;
      cf.out = X.out;
      cf.out_cap = X.cap;
      cf.label = parent;
      cf.giant_bits = gbits;
      cf.giant_count = &c->ds->giant_count;
      cf.pivot_dev = &piv[k];
      cf.n = n;
      cf.best = best;  // the survivors are expected to be sparse (Theorem 1)
      cf.kl = kl;
      record_ends(cf);
      cf.st = next_scan(c, CNT_LVL + LVL_MAX + k);
      // the pass streams the whole list; the method reads only its heavy
      // edges (the list less its light list k+1)
      const double per = E[k].id ? 16.0 : 12.0;
      const double fixed = k == 0 ? per * (double)m0 : 0.0;
      PROF_TERMS(MST_K_FILTER, fixed, fixed, launch_compact(CM_FILTER, cf, caps[k], s),
                 ProfTerm{k == 0 ? -1 : CNT_LVL + k, per, per}, ProfTerm{CNT_LVL + k + 1, 0.0, -per},
                 ProfTerm{CNT_LVL + LVL_MAX + k, 16.0, 16.0});
      TRY(boruvka_planned(X, Y, CNT_LVL + LVL_MAX + k, cur_u != nullptr, exec));
    }
    return MST_OK;
  }

  // Back to the state init() left (the host-driven path after a plan that
  // did not hold).
  mst_status restart() {
    CK(cudaMemsetAsync(best, 0xff, (size_t)n * 8, s));
    launch_iota(parent, n, c->sms, s);
    CK(cudaMemsetAsync(bits, 0, (m + 31) / 32 * 4, s));
    TRY(clear_device_flags(c, s));
    CK(cudaMemsetAsync(c->wsum, 0, WSUM_SLOTS * sizeof(u64), s));
    c->pivot_counter = 0;
    rounds = 0;
    return MST_OK;
  }

  // The ids come from the chosen-edge bitmap; the total from the counters the
  // hooking kernels added each chosen edge's weight into (no gather of w).
  mst_status finalize(uint32_t *out_ids, uint32_t *out_count, u64 *total_weight, uint32_t tolerated = 0) {
    PROF(MST_K_FINALIZE, (double)((m + 31) / 32 * 4), CNT_AUX, 4.0, -1, 0.0,
         launch_finalize(bits, m, nullptr, out_ids, out_count, total_weight, next_scan(c, CNT_AUX), s);
         launch_wsum_total(c->wsum, total_weight, s));
    return readback(c, s, tolerated);
  }
};

bool use_filter(const mst_config &cfg, uint32_t n, uint64_t m) {
  if (cfg.variant == MST_VARIANT_FILTER) return true;
  if (cfg.variant == MST_VARIANT_BORUVKA) return false;
  return m >= (1ULL << 20) && 2.0 * (double)m > 8.0 * (double)n;
}

mst_status solve_device(mst_ctx *c, uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                        const uint32_t *w, uint32_t *out_ids, uint32_t *out_count, u64 *total_weight,
                        cudaStream_t s) {
  if (m >= (1ULL << 32)) return MST_ERR_TOO_LARGE;
  if (!out_count || !total_weight || (m > 0 && (!src || !dst || !w || !out_ids))) return MST_ERR_INVALID_ARG;
  if (!aligned4(src) || !aligned4(dst) || !aligned4(w) || !aligned4(out_ids)) return MST_ERR_INVALID_ARG;
  if (n == 0 || m == 0) {
    if (m > 0 && n == 0) return MST_ERR_VERTEX_RANGE;
    CK(cudaMemsetAsync(out_count, 0, sizeof(uint32_t), s));
    CK(cudaMemsetAsync(total_weight, 0, sizeof(u64), s));
    CK(cudaStreamSynchronize(s));
    return MST_OK;
  }
  Solve S(c, s, n, m);
  TRY(S.init());
  ++c->solves;
  S.src = src;
  S.dst = dst;
  S.w_in = w;
  const EdgeList in{src, dst, w, nullptr};
  c->pivot_counter = 0;
  const bool filt = use_filter(c->cfg, n, m);
  ListBuf local;
  uint64_t m_local = 0;
  bool applied = false;
  TRY(S.tile_preprocess(w, !filt, local, m_local, applied));
  if (applied) {  // continue on the contracted graph (ids already validated)
    if (filt)
      TRY(S.filter(local.list(), m_local, false, 0, false, true));
    else
      TRY(S.boruvka(local.list(), m_local, false, true, true));
  } else if (filt) {
    if (S.plan_eligible()) {
      bool planned = false;
      TRY(S.filter_planned(planned));
      if (planned) {
        ++c->planned;
        constexpr uint32_t replan = ERR_OVERFLOW | ERR_HANDBACK;
        TRY(S.finalize(out_ids, out_count, total_weight, replan));
        if (!(c->hs->err & replan) && !c->hs->jump_flag) return MST_OK;
        ++c->plan_fallbacks;
      }
      TRY(S.restart());
    }
    TRY(S.filter(in, m, true, 0));
  } else {
    TRY(S.boruvka(in, m, true));
  }
  return S.finalize(out_ids, out_count, total_weight);
}

mst_status validate_cfg(const mst_config *cfg) {
  if (cfg->variant < 0 || cfg->variant > 2) return MST_ERR_INVALID_ARG;
  if (cfg->dedupe != MST_DEDUPE_AUTO && cfg->dedupe != MST_DEDUPE_HASH && cfg->dedupe != MST_DEDUPE_NONE &&
      cfg->dedupe != MST_DEDUPE_SORT)
    return MST_ERR_INVALID_ARG;
  if (cfg->pivot_sample == 0 || cfg->pivot_sample > (1u << 24)) return MST_ERR_INVALID_ARG;
  if (!(cfg->filter_max_avg_degree > 0.0f)) return MST_ERR_INVALID_ARG;
  if (cfg->tile_contract < -1 || cfg->tile_contract > 1) return MST_ERR_INVALID_ARG;
  if (cfg->base_case < 0 || cfg->base_case > 1) return MST_ERR_INVALID_ARG;
  if (cfg->graph_rounds < 0 || cfg->graph_rounds > 1) return MST_ERR_INVALID_ARG;
  if (cfg->graph_jump_launches < 1 || cfg->graph_jump_launches > 8) return MST_ERR_INVALID_ARG;
  if (cfg->filter_carry < 0 || cfg->filter_carry > 1) return MST_ERR_INVALID_ARG;
  if (cfg->filter_split < 0 || cfg->filter_split > 1) return MST_ERR_INVALID_ARG;
  if (cfg->min_edges_sort < 0 || cfg->min_edges_sort > 1) return MST_ERR_INVALID_ARG;
  if (cfg->jump_steps < 1 || cfg->jump_steps > 4096) return MST_ERR_INVALID_ARG;
  if (cfg->tile_filter < 0 || cfg->tile_filter > 1) return MST_ERR_INVALID_ARG;
  if (cfg->tile_vertices < 32 || cfg->tile_vertices > 4096) return MST_ERR_INVALID_ARG;
  if (cfg->spin_limit < 1) return MST_ERR_INVALID_ARG;
  if (shape_index(cfg->block_threads, cfg->items_per_thread) < 0) return MST_ERR_INVALID_ARG;
  if (cfg->filter_plan < 0 || cfg->filter_plan > 1) return MST_ERR_INVALID_ARG;
  if (relabel_shape_index(cfg->relabel_block_threads, cfg->relabel_items_per_thread) < 0) return MST_ERR_INVALID_ARG;
  if (!(cfg->pivot_quantile >= 1.0f / 64.0f && cfg->pivot_quantile <= 0.5f)) return MST_ERR_INVALID_ARG;
  return MST_OK;
}

mst_status ensure_sample(mst_ctx *c) {
  if (c->sample_cap >= c->cfg.pivot_sample) return MST_OK;
  if (c->sample_buf) cudaFree(c->sample_buf);
  c->sample_buf = nullptr;
  c->sample_cap = 0;
  if (cudaMalloc(&c->sample_buf, (size_t)c->cfg.pivot_sample * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return MST_ERR_OOM;
  }
  c->sample_cap = c->cfg.pivot_sample;
  return MST_OK;
}

mst_status record(mst_ctx *c, mst_status st) {
  if (st == MST_ERR_CUDA) {
    const int e = (int)cudaGetLastError();
    c->last_cuda = tl_cuda_error ? tl_cuda_error : e;
    c->last_cuda_line = tl_cuda_error ? tl_cuda_line : 0;
  }
  tl_cuda_error = 0;
  tl_cuda_line = 0;
  c->last = st;
  return st;
}

// MST_ERR_CUDA from a call checked in place (not through CK).
mst_status record_cuda(mst_ctx *c, int line) {
  const int e = (int)cudaGetLastError();
  tl_cuda_error = e ? e : (int)cudaErrorUnknown;
  tl_cuda_line = line;
  return record(c, MST_ERR_CUDA);
}

// ---------------------------------------------------------------- batched

// Graph of union position e: the largest g with off[g] <= e (graphs are
// contiguous ranges of positions; empty graphs are passed over).
__device__ __forceinline__ uint32_t batch_graph_of(const uint64_t *off, uint32_t G, uint64_t e) {
  uint32_t lo = 0, hi = G;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (off[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// The batched size tables, read on the device: vert_off[g] = n[0] + ... +
// n[g-1] (g = 0..G, an exclusive scan in one block), totals[0] = all vertices,
// totals[1] = edge_off[G] (all edges); ERR_TABLE if edge_off[0] != 0 or the
// offsets decrease somewhere.
constexpr int TAB_THREADS = 1024;
__global__ void __launch_bounds__(TAB_THREADS) batch_tables_kernel(const uint32_t *gn, const uint64_t *edge_off,
                                                                  uint32_t G, uint64_t *vert_off, u64 *totals,
                                                                  uint32_t *err) {
  __shared__ u64 s_warp[TAB_THREADS / 32];
  __shared__ u64 s_carry;
  __shared__ uint32_t s_bad;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_carry = 0;
    s_bad = edge_off[0] != 0 ? 1u : 0u;
  }
  __syncthreads();
  for (uint64_t base = 0; base < G; base += TAB_THREADS) {
    const uint64_t g = base + threadIdx.x;
    const u64 x = g < G ? (u64)gn[g] : 0ULL;
    if (g < G && edge_off[g + 1] < edge_off[g]) atomicOr(&s_bad, 1u);
    u64 incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const u64 v = s_warp[lane];
      u64 wi = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, wi, d);
        if (lane >= d) wi += y;
      }
      s_warp[lane] = wi - v;  // exclusive prefix of the warps' sums
    }
    __syncthreads();
    const u64 excl = s_carry + s_warp[wid] + incl - x;
    if (g < G) vert_off[g] = excl;
    __syncthreads();  // every thread has read s_carry and s_warp
    if (threadIdx.x == TAB_THREADS - 1) s_carry = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    vert_off[G] = s_carry;
    totals[0] = s_carry;
    totals[1] = edge_off[G];
    if (s_bad) atomicOr(err, ERR_TABLE);
  }
}

// Union vertex ids: edge e of graph g gets its ends offset by vert_off[g].
// Each block takes a contiguous chunk of edges (so a thread walks forward
// through few graphs), independent of how the edges split into graphs.
__global__ void batch_offset_kernel(const uint32_t *src, const uint32_t *dst, const uint64_t *edge_off,
                                    const uint64_t *vert_off, uint32_t *usrc, uint32_t *udst, const uint32_t *gn,
                                    uint32_t G, uint64_t m, uint32_t *err) {
  const uint64_t chunk = ((m + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = min(m, lo + chunk);
  uint64_t e = lo + threadIdx.x;
  if (e >= hi) return;
  uint32_t g = batch_graph_of(edge_off, G, e);
  for (; e < hi; e += blockDim.x) {
    while (edge_off[g + 1] <= e) ++g;
    const uint32_t vo = (uint32_t)vert_off[g], ng = gn[g];
    const uint32_t a = src[e], b = dst[e];
    if (a >= ng || b >= ng) atomicOr(err, ERR_VERTEX);
    usrc[e] = a < ng ? a + vo : vo;
    udst[e] = b < ng ? b + vo : vo;
  }
}

// Segment offsets of the per-graph forests in the ascending union ids:
// msf_off[g] = number of union ids below edge_off[g] (g = 0..G).
__global__ void batch_seg_kernel(const uint32_t *ids, const uint32_t *count, const uint64_t *edge_off, uint32_t G,
                                 uint64_t *msf_off) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > G) return;
  const uint64_t target = edge_off[g];
  uint64_t lo = 0, hi = *count;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    if ((uint64_t)ids[mid] < target)
      lo = mid + 1;
    else
      hi = mid;
  }
  msf_off[g] = lo;
}

// Graph-local ids and per-graph weight sums (total_weight zeroed before).
// Contiguous chunks per block; a warp adds up the weights of each run of ids
// of one graph and issues one atomic per run.
__global__ void batch_split_kernel(const uint32_t *ids, const uint32_t *count, const uint64_t *edge_off, uint32_t G,
                                   const uint32_t *w, uint32_t *out_ids, u64 *total_weight) {
  const uint64_t k = *count;
  const uint64_t chunk = ((k + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = min(k, lo + chunk);
  const int lane = threadIdx.x & 31;
  uint32_t g = 0;
  bool first = true;
  for (uint64_t b0 = lo; b0 < hi; b0 += blockDim.x) {  // warp-uniform trip count
    const uint64_t i = b0 + threadIdx.x;
    const bool in = i < hi;
    u64 v = 0;
    uint32_t gi = 0xffffffffu;
    if (in) {
      const uint32_t id = ids[i];
      if (first) {
        g = batch_graph_of(edge_off, G, id);
        first = false;
      }
      while (edge_off[g + 1] <= id) ++g;
      out_ids[i] = (uint32_t)((uint64_t)id - edge_off[g]);
      v = w[id];
      gi = g;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {  // segmented inclusive sum over runs of equal graph
      const u64 pv = __shfl_up_sync(0xffffffffu, v, o);
      const uint32_t pg = __shfl_up_sync(0xffffffffu, gi, o);
      if (lane >= o && pg == gi) v += pv;
    }
    const uint32_t ng = __shfl_down_sync(0xffffffffu, gi, 1);
    if (in && (lane == 31 || ng != gi)) atomicAdd(total_weight + gi, v);
  }
}

}  // namespace

// A device buffer of the host entry points of at least `bytes`, grown (after
// the device is idle, since the old one may still be read) when too small.
static mst_status host_side_buffer(void *&buf, size_t &cap, size_t bytes) {
  if (cap >= bytes && buf) return MST_OK;
  CK(cudaDeviceSynchronize());
  if (buf) cudaFree(buf);
  buf = nullptr;
  cap = 0;
  const size_t want = bytes < 256 ? 256 : bytes;
  if (cudaMalloc(&buf, want) != cudaSuccess) {
    cudaGetLastError();
    return MST_ERR_OOM;
  }
  cap = want;
  return MST_OK;
}

// The forest size and weight of a solve, read back through the handle's
// page-locked words.  A copy into pageable host memory is synchronous and
// staged by the driver, and it can queue behind a large host-to-device copy
// in flight on another stream (the next graph's input in
// mst_solve_host_many), which would serialise copy and solve.
static mst_status read_size_and_weight(mst_ctx *c, const uint32_t *d_count, const u64 *d_total, cudaStream_t s,
                                uint32_t &cnt, uint64_t &total) {
  CK(cudaMemcpyAsync(&c->hres[0], d_count, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&c->hres[1], d_total, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cnt = (uint32_t)(c->hres[0] & 0xffffffffu);
  total = c->hres[1];
  return MST_OK;
}

// ===================================================================== ABI

extern "C" {

void mst_config_default(mst_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->variant = MST_VARIANT_BORUVKA;
  cfg->dedupe = MST_DEDUPE_AUTO;
  cfg->tile_contract = 0;
  cfg->tile_vertices = 1024;
  cfg->pivot_sample = 1u << 16;
  cfg->seed = 0x2302121990ULL;
  cfg->filter_min_edges = 1ULL << 20;
  // measured on GB300 (the paper uses 4 on its cluster): with median pivots RMAT n=2^24 m=2^28 took 9.72 /
  // 9.42 / 9.40 / 9.42 / 9.60 ms at 0.9 / 1.0 / 1.1 / 1.5 / 2.0, and with the default 1/8-quantile pivots
  // 5.26 / 5.28 / 5.27 ms at 0.75 / 1.25 / 2.5 (the lists 2^28 -> 2^25 -> 2^22 stop at the same level).
  cfg->filter_max_avg_degree = 1.25f;
  cfg->base_case = 1;
  cfg->graph_rounds = 1;
  cfg->graph_jump_launches = 2;
  cfg->filter_carry = 0;  // measured slower on GB300 (the merged tail loses the fused minEdges)
  cfg->filter_split = 0;
  cfg->min_edges_sort = 0;
  cfg->jump_steps = 64;
  cfg->tile_filter = 0;  // measured slower on GB300: the light phase adds synchronised rounds in each tile
  cfg->spin_limit = 1u << 21;  // about a second of polling at the measured poll rate
  cfg->block_threads = 0;      // 0: 256 threads per block
  cfg->items_per_thread = 0;   // 0: 8 edges per thread
  cfg->filter_plan = 1;
  cfg->relabel_block_threads = 0;     // 0 and 0: 128 x 4
  cfg->relabel_items_per_thread = 0;
  // Alg. 2 splits at the sample median; on GB300 a split at the 1/8 quantile measured fastest (RMAT n=2^24
  // m=2^28: 7.16 ms at 1/2, 5.54 at 1/4, 5.25 at 1/8, 5.35 at 1/16): light lists an eighth as long and two
  // partition levels instead of five, for the same total of filtered heavy edges.
  cfg->pivot_quantile = 0.125f;
}

const char *mst_status_string(mst_status s) {
  switch (s) {
    case MST_OK: return "ok";
    case MST_ERR_INVALID_ARG: return "invalid argument";
    case MST_ERR_VERTEX_RANGE: return "vertex id out of range";
    case MST_ERR_TOO_LARGE: return "graph too large (m >= 2^32)";
    case MST_ERR_OOM: return "out of device memory";
    case MST_ERR_CUDA: return "CUDA runtime error";
    case MST_ERR_INTERNAL: return "internal error (bounded device loop exhausted)";
    case MST_ERR_NOT_SUPPORTED: return "not supported";
  }
  return "unknown status";
}

mst_status mst_create(mst_handle *out, const mst_config *cfg) {
  if (!out) return MST_ERR_INVALID_ARG;
  *out = nullptr;
  mst_config def;
  mst_config_default(&def);
  if (!cfg) cfg = &def;
  if (validate_cfg(cfg) != MST_OK) return MST_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return MST_ERR_CUDA;
  }
  mst_ctx *c = new (std::nothrow) mst_ctx();
  if (!c) return MST_ERR_OOM;
  c->cfg = *cfg;
  c->device = cfg->device;
  DeviceGuard g(c->device);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = c->device;
  bool ok = cudaMemPoolCreate(&c->pool, &props) == cudaSuccess;
  if (ok) {
    uint64_t thr = ~0ULL;
    ok = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&c->ds, sizeof(DevState)) == cudaSuccess;
  ok = ok && cudaMemset(c->ds, 0, sizeof(DevState)) == cudaSuccess;
  ok = ok && cudaHostAlloc(&c->hs, sizeof(DevState), cudaHostAllocMapped) == cudaSuccess;
  ok = ok && cudaHostGetDevicePointer((void **)&c->hs_dev, c->hs, 0) == cudaSuccess;
  ok = ok && cudaHostAlloc(&c->hflag, 64, cudaHostAllocMapped) == cudaSuccess;
  ok = ok && cudaHostGetDevicePointer((void **)&c->hflag_dev, c->hflag, 0) == cudaSuccess;
  if (ok) *c->hflag = 0;
  ok = ok && cudaMallocHost(&c->hres, 2 * sizeof(u64)) == cudaSuccess;
  ok = ok && ensure_sample(c) == MST_OK;
  ok = ok && cudaMalloc(&c->pivot_scratch, pivot_scratch_bytes()) == cudaSuccess;
  ok = ok && cudaMalloc(&c->wsum, WSUM_SLOTS * sizeof(u64)) == cudaSuccess;
  ok = ok && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mst_destroy(c);
    return MST_ERR_CUDA;
  }
  *out = c;
  return MST_OK;
}

void mst_destroy(mst_handle h) {
  if (!h) return;
  {
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    if (h->ds) cudaFree(h->ds);
    if (h->hs) cudaFreeHost(h->hs);
    if (h->hflag) cudaFreeHost(h->hflag);
    if (h->hres) cudaFreeHost(h->hres);
    for (int k = 0; k < 2; ++k)
      if (h->hin[k]) cudaFree(h->hin[k]);
    if (h->hout) cudaFree(h->hout);
    if (h->rl_mem) cudaFree(h->rl_mem);
    if (h->status) cudaFree(h->status);
    if (h->sample_buf) cudaFree(h->sample_buf);
    if (h->pivot_scratch) cudaFree(h->pivot_scratch);
    if (h->wsum) cudaFree(h->wsum);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (int k = 0; k < 2; ++k) {
      if (h->in_ready[k]) cudaEventDestroy(h->in_ready[k]);
      if (h->in_free[k]) cudaEventDestroy(h->in_free[k]);
    }
    for (auto &rg : h->round_graphs) {
      cudaGraphExecDestroy(rg.exec);
      cudaGraphDestroy(rg.graph);
    }
    if (h->grounds) cudaFree(h->grounds);
    if (h->pool) cudaMemPoolDestroy(h->pool);
    for (auto &r : h->prof_pending) {
      if (r.a) h->ev_pool.push_back(r.a);
      if (r.b) h->ev_pool.push_back(r.b);
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    cudaGetLastError();
  }
  delete h;
}

mst_status mst_set_config(mst_handle h, const mst_config *cfg) {
  if (!h || !cfg) return MST_ERR_INVALID_ARG;
  if (validate_cfg(cfg) != MST_OK || cfg->device != h->device) return record(h, MST_ERR_INVALID_ARG);
  DeviceGuard g(h->device);
  h->cfg = *cfg;
  return record(h, ensure_sample(h));
}

mst_status mst_get_error(mst_handle h, void *stream) {
  if (!h) return MST_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return record_cuda(h, __LINE__);
  const mst_status dev = readback(h, (cudaStream_t)stream);  // flags the device latched since the last call began
  return h->last != MST_OK ? h->last : dev;
}

int mst_last_cuda_error(mst_handle h, int *line) {
  if (line) *line = h ? h->last_cuda_line : 0;
  return h ? h->last_cuda : 0;
}

mst_status mst_profile_enable(mst_handle h, int enable) {
  if (!h) return MST_ERR_INVALID_ARG;
  h->prof_on = enable != 0;
  if (h->prof_on) std::memset(h->prof, 0, sizeof(h->prof));
  return MST_OK;
}

mst_status mst_profile_classes(mst_handle h, uint32_t mask) {
  if (!h) return MST_ERR_INVALID_ARG;
  h->prof_mask = mask;
  return MST_OK;
}

mst_status mst_profile_get(mst_handle h, int kind, mst_kernel_stats *out) {
  if (!h || !out || kind < 0 || kind >= MST_K_COUNT) return MST_ERR_INVALID_ARG;
  *out = h->prof[kind];
  return MST_OK;
}

mst_status mst_host_counters_get(mst_handle h, mst_host_counters *out) {
  if (!h || !out) return MST_ERR_INVALID_ARG;
  out->solves = h->solves;
  out->readbacks = h->readbacks;
  out->planned = h->planned;
  out->plan_fallbacks = h->plan_fallbacks;
  return MST_OK;
}

uint64_t mst_workspace_bytes(uint32_t n, uint64_t m, const mst_config *cfg) {
  mst_config def;
  mst_config_default(&def);
  if (!cfg) cfg = &def;
  const uint64_t vert = (uint64_t)n * (8 + 4 + 4 + 4);  // best, parent, two active lists
  const uint64_t bits = (m + 31) / 32 * 4;
  const uint64_t list = 16 * m + 1024;
  uint64_t edges = 2 * (list + list / 4 + (16ULL << 16));       // the handle's ping-pong round lists (grown with
                                                                 // a quarter of headroom, in steps of 2^16 edges)
  if (cfg->dedupe != MST_DEDUPE_NONE) edges += list + 32 * m + 16384;  // dedupe list + hash table
  if (cfg->variant != MST_VARIANT_BORUVKA) edges += 2 * list;   // partition levels and filtered lists
  return vert + bits + edges;
}

mst_status mst_solve(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                     const uint32_t *d_w, uint32_t *d_msf_ids, uint32_t *d_msf_count, uint64_t *d_total_weight,
                     void *stream) {
  if (!h) return MST_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  return record(h, solve_device(h, n, m, d_src, d_dst, d_w, d_msf_ids, d_msf_count, (u64 *)d_total_weight,
                                (cudaStream_t)stream));
}

mst_status mst_solve_host(mst_handle h, uint32_t n, uint64_t m, const uint32_t *h_src, const uint32_t *h_dst,
                          const uint32_t *h_w, uint32_t *h_msf_ids, uint32_t *h_msf_count, uint64_t *h_total_weight,
                          void *stream) {
  if (!h) return MST_ERR_INVALID_ARG;
  if (!h_msf_count || !h_total_weight || (m > 0 && (!h_src || !h_dst || !h_w || !h_msf_ids)))
    return record(h, MST_ERR_INVALID_ARG);
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t cap = m < (uint64_t)(n > 0 ? n - 1 : 0) ? m : (uint64_t)(n > 0 ? n - 1 : 0);
  const uint64_t stride = round_up(m * 4 + 16, 256);
  mst_status st = host_side_buffer(h->hin[0], h->hin_cap[0], stride * 3);
  if (st == MST_OK) st = host_side_buffer(h->hout, h->hout_cap, cap * 4 + 256);
  if (st != MST_OK) return record(h, st);
  char *b = static_cast<char *>(h->hin[0]);
  uint32_t *d_src = (uint32_t *)b, *d_dst = (uint32_t *)(b + stride), *d_w = (uint32_t *)(b + 2 * stride);
  uint32_t *d_out = static_cast<uint32_t *>(h->hout);
  uint32_t *d_count = (uint32_t *)((char *)d_out + cap * 4);
  u64 *d_total = (u64 *)((char *)d_out + round_up(cap * 4 + 4, 8));
  if (m > 0) {
    if (cudaMemcpyAsync(d_src, h_src, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_dst, h_dst, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_w, h_w, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return record_cuda(h, __LINE__);
  }
  st = solve_device(h, n, m, d_src, d_dst, d_w, d_out, d_count, d_total, s);
  if (st != MST_OK) return record(h, st);
  uint32_t cnt = 0;
  if (read_size_and_weight(h, d_count, d_total, s, cnt, *h_total_weight) != MST_OK) return record_cuda(h, __LINE__);
  *h_msf_count = cnt;
  if (cnt > 0 && (cudaMemcpyAsync(h_msf_ids, d_out, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess))
    return record_cuda(h, __LINE__);
  return record(h, MST_OK);
}

mst_status mst_solve_host_many(mst_handle h, uint32_t count, mst_host_graph *gs, void *stream) {
  if (!h) return MST_ERR_INVALID_ARG;
  if (count == 0) return record(h, MST_OK);
  if (!gs) return record(h, MST_ERR_INVALID_ARG);
  uint64_t max_m = 0, max_cap = 0;
  for (uint32_t i = 0; i < count; ++i) {
    gs[i].status = MST_ERR_INTERNAL;
    gs[i].msf_count = 0;
    gs[i].total_weight = 0;
  }
  for (uint32_t i = 0; i < count; ++i) {
    const mst_host_graph &g = gs[i];
    if (g.m > 0 && (!g.src || !g.dst || !g.w || !g.msf_ids)) return record(h, gs[i].status = MST_ERR_INVALID_ARG);
    if (g.m >= (1ULL << 32)) return record(h, gs[i].status = MST_ERR_TOO_LARGE);
    const uint64_t cap = g.m < (uint64_t)(g.n > 0 ? g.n - 1 : 0) ? g.m : (uint64_t)(g.n > 0 ? g.n - 1 : 0);
    max_m = std::max(max_m, g.m);
    max_cap = std::max(max_cap, cap);
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!h->copy_stream && cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return record_cuda(h, __LINE__);
  for (int k = 0; k < 2; ++k) {
    if (!h->in_ready[k] && cudaEventCreateWithFlags(&h->in_ready[k], cudaEventDisableTiming) != cudaSuccess)
      return record_cuda(h, __LINE__);
    if (!h->in_free[k] && cudaEventCreateWithFlags(&h->in_free[k], cudaEventDisableTiming) != cudaSuccess)
      return record_cuda(h, __LINE__);
  }
  const uint64_t stride = round_up(max_m * 4 + 16, 256);
  mst_status st = MST_OK;
  for (int k = 0; k < 2 && st == MST_OK; ++k) st = host_side_buffer(h->hin[k], h->hin_cap[k], stride * 3);
  if (st == MST_OK) st = host_side_buffer(h->hout, h->hout_cap, max_cap * 4 + 256);
  if (st != MST_OK) return record(h, gs[0].status = st);
  // both input sets count as free (for the copy stream) once s reaches this
  // point: earlier work of this handle on s may still read them
  for (int k = 0; k < 2; ++k)
    if (cudaEventRecord(h->in_free[k], s) != cudaSuccess) return record_cuda(h, __LINE__);
  uint32_t *d_out = static_cast<uint32_t *>(h->hout);
  uint32_t *d_count = (uint32_t *)((char *)d_out + max_cap * 4);
  u64 *d_total = (u64 *)((char *)d_out + round_up(max_cap * 4 + 4, 8));
  auto set_of = [&](uint32_t i, int a) { return (uint32_t *)(static_cast<char *>(h->hin[i % 2]) + (size_t)a * stride); };
  auto issue_copy = [&](uint32_t i) -> bool {
    const int k = (int)(i % 2);
    if (cudaStreamWaitEvent(h->copy_stream, h->in_free[k], 0) != cudaSuccess) return false;
    const mst_host_graph &g = gs[i];
    if (g.m > 0) {
      const uint32_t *srcs[3] = {g.src, g.dst, g.w};
      for (int a = 0; a < 3; ++a)
        if (cudaMemcpyAsync(set_of(i, a), srcs[a], g.m * 4, cudaMemcpyHostToDevice, h->copy_stream) != cudaSuccess)
          return false;
    }
    return cudaEventRecord(h->in_ready[k], h->copy_stream) == cudaSuccess;
  };
  mst_status first = MST_OK;
  if (!issue_copy(0)) return record_cuda(h, __LINE__);
  uint32_t i = 0;
  for (; i < count; ++i) {
    const int k = (int)(i % 2);
    if (i + 1 < count && !issue_copy(i + 1)) {  // overlaps the solve below
      st = record_cuda(h, __LINE__);
      break;
    }
    if (cudaStreamWaitEvent(s, h->in_ready[k], 0) != cudaSuccess) {
      st = record_cuda(h, __LINE__);
      break;
    }
    mst_host_graph &g = gs[i];
    st = solve_device(h, g.n, g.m, set_of(i, 0), set_of(i, 1), set_of(i, 2), d_out, d_count, d_total, s);
    if (cudaEventRecord(h->in_free[k], s) != cudaSuccess) {
      st = record_cuda(h, __LINE__);
      break;
    }
    if (st == MST_OK) {
      uint32_t cnt = 0;
      uint64_t tot = 0;
      if (read_size_and_weight(h, d_count, d_total, s, cnt, tot) != MST_OK ||
          (cnt > 0 && (cudaMemcpyAsync(g.msf_ids, d_out, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaStreamSynchronize(s) != cudaSuccess))) {
        st = record_cuda(h, __LINE__);
        g.status = st;
        if (first == MST_OK) first = st;
        ++i;
        break;
      }
      g.msf_count = cnt;
      g.total_weight = tot;
    }
    g.status = st;
    if (st != MST_OK && first == MST_OK) first = st;
    if (st == MST_ERR_CUDA || st == MST_ERR_OOM) {
      ++i;
      break;
    }
  }
  // a copy issued for a graph that was not solved must finish before the
  // buffers are used again (each event marks the last copy into its buffer)
  for (int k = 0; k < 2; ++k) cudaStreamWaitEvent(s, h->in_ready[k], 0);
  if (st == MST_ERR_CUDA && first == MST_OK) first = st;
  return record(h, first);
}

mst_status mst_solve_batched(mst_handle h, uint32_t num_graphs, const uint32_t *d_n, const uint64_t *d_edge_off,
                             const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w, uint32_t *d_msf_ids,
                             uint64_t *d_msf_off, uint64_t *d_total_weight, void *stream) {
  if (!h) return MST_ERR_INVALID_ARG;
  if (num_graphs == 0) return record(h, MST_OK);
  if (!d_n || !d_edge_off || !d_msf_off || !d_total_weight) return record(h, MST_ERR_INVALID_ARG);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  // vertex offsets of the disjoint union and the totals, from the device tables
  Buf voff_b;
  mst_status st = voff_b.alloc(h, ((size_t)num_graphs + 1) * 8, s);
  if (st != MST_OK) return record(h, st);
  uint64_t *d_voff = voff_b.as<uint64_t>();
  if (clear_device_flags(h, s) != MST_OK) return record_cuda(h, __LINE__);
  batch_tables_kernel<<<1, TAB_THREADS, 0, s>>>(d_n, d_edge_off, num_graphs, d_voff, &h->ds->count[CNT_AUX],
                                                &h->ds->err);
  st = readback(h, s);
  if (st != MST_OK) return record(h, st);
  const uint64_t n_total = h->hs->count[CNT_AUX], m = h->hs->count[CNT_AUX + 1];
  if (n_total >= (1ULL << 32) || m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  if (m > 0 && (!d_src || !d_dst || !d_w || !d_msf_ids)) return record(h, MST_ERR_INVALID_ARG);
  const uint32_t n = (uint32_t)n_total;
  // union endpoints, union ids
  Buf uni_b, ids_b;
  const uint64_t stride = round_up(m * 4 + 16, 256);
  st = uni_b.alloc(h, stride * 2, s);
  const uint64_t cap = m < (uint64_t)n ? m : (uint64_t)n;
  // ids, then (256-byte aligned) the forest size, then 256 bytes on, its weight
  if (st == MST_OK) st = ids_b.alloc(h, round_up(cap * 4, 256) + 512, s);
  if (st != MST_OK) return record(h, st);
  uint32_t *usrc = uni_b.as<uint32_t>(), *udst = (uint32_t *)((char *)uni_b.p + stride);
  uint32_t *ids = ids_b.as<uint32_t>();
  uint32_t *d_count = (uint32_t *)((char *)ids + round_up(cap * 4, 256));
  u64 *d_sum = (u64 *)((char *)d_count + 256);
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((m + 2047) / 2048, (uint64_t)h->sms * 8));
  if (m > 0)
    batch_offset_kernel<<<grid, 256, 0, s>>>(d_src, d_dst, d_edge_off, d_voff, usrc, udst, d_n, num_graphs, m,
                                             &h->ds->err);
  st = readback(h, s);
  if (st != MST_OK) return record(h, st);
  st = solve_device(h, n, m, usrc, udst, d_w, ids, d_count, d_sum, s);
  if (st != MST_OK) return record(h, st);
  if (cudaMemsetAsync(d_total_weight, 0, (size_t)num_graphs * 8, s) != cudaSuccess) return record_cuda(h, __LINE__);
  batch_seg_kernel<<<(num_graphs + 1 + 255) / 256, 256, 0, s>>>(ids, d_count, d_edge_off, num_graphs, d_msf_off);
  const unsigned sgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((cap + 2047) / 2048, (uint64_t)h->sms * 8));
  batch_split_kernel<<<sgrid, 256, 0, s>>>(ids, d_count, d_edge_off, num_graphs, d_w, d_msf_ids, (u64 *)d_total_weight);
  if (cudaStreamSynchronize(s) != cudaSuccess) return record_cuda(h, __LINE__);
  return record(h, MST_OK);
}

// ---------------------------------------------------------------- steps

mst_status mst_step_min_edges(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                              const uint32_t *d_w, const uint32_t *d_id, uint64_t *d_best, void *stream) {
  if (!h || !d_best || (m > 0 && (!d_u || !d_v || !d_w))) return MST_ERR_INVALID_ARG;
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_best, 0xff, (size_t)n * 8, s) != cudaSuccess ||
      cudaMemsetAsync(&h->ds->err, 0, 4, s) != cudaSuccess)
    return record_cuda(h, __LINE__);
  launch_min_edges(EdgeList{d_u, d_v, d_w, d_id}, m, n, 1, KeyLayout{0, 0, 0}, (u64 *)d_best, &h->ds->err, h->sms, s);
  return record(h, readback(h, s));
}

mst_status mst_step_contract(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                             const uint32_t *d_w, const uint32_t *d_id, uint32_t *d_parent, uint32_t *d_chosen,
                             void *stream) {
  if (!h || !d_parent || !d_chosen || d_id || (m > 0 && (!d_u || !d_v || !d_w))) return MST_ERR_INVALID_ARG;
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  Solve S(h, s, n, m);
  mst_status st = S.init(d_parent, d_chosen);
  if (st != MST_OK) return record(h, st);
  S.src = d_u;
  S.dst = d_v;
  const EdgeList E{d_u, d_v, d_w, nullptr};
  launch_min_edges(E, m, n, 1, S.kl, S.best, &h->ds->err, h->sms, s);
  if (zero_counters(h, s) != MST_OK) return record_cuda(h, __LINE__);
  HookArgs ha{};
  ha.shape = shape_index(h->cfg.block_threads, h->cfg.items_per_thread);
  ha.ncand = n;
  ha.best = S.best;
  ha.kl = S.kl;
  ha.src = d_u;
  ha.dst = d_v;
  ha.parent = d_parent;
  ha.chosen_bits = d_chosen;
  ha.active_out = S.act[0];
  ha.counter = &h->ds->count[CNT_ACTIVE];
  ha.err = &h->ds->err;
  ha.wsum = h->wsum;
  launch_hook(ha, n, s);
  return record(h, S.jump_until_stars(S.act[0], &h->ds->count[CNT_ACTIVE], 0, n, 1));
}

static mst_status step_compact(mst_handle h, CompactMode mode, uint32_t n, uint64_t m, const uint32_t *d_u,
                               const uint32_t *d_v, const uint32_t *d_w, const uint32_t *d_id, const uint32_t *label,
                               uint64_t pivot, uint32_t *d_ou, uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid,
                               uint64_t *d_out_count, void *stream) {
  if (!h || !d_out_count || (m > 0 && (!d_u || !d_v || !d_w || !d_ou || !d_ov || !d_ow || !d_oid)))
    return MST_ERR_INVALID_ARG;
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  mst_status st = ensure_status(h, m, s);
  if (st != MST_OK) return record(h, st);
  if (clear_device_flags(h, s) != MST_OK) return record_cuda(h, __LINE__);
  const EdgeList E{d_u, d_v, d_w, d_id};
  CompactArgs a{};
  a.shape = mode == CM_RELABEL ? relabel_shape_index(h->cfg.relabel_block_threads, h->cfg.relabel_items_per_thread)
                               : shape_index(h->cfg.block_threads, h->cfg.items_per_thread);
  a.warp_partition = h->cfg.pivot_quantile <= 0.125f ? 1 : 0;  // the solves' choice for this configuration
  a.in = E;
  a.m = m;
  a.out = EdgeOut{d_ou, d_ov, d_ow, d_oid};
  a.label = label;
  a.pivot = pivot;
  a.n = n;
  a.validate = (mode == CM_RELABEL || mode == CM_FILTER) ? 1 : 0;
  Buf table_b, giant_b;
  if (mode == CM_FILTER && n > 0 && m > 0) {  // the solver's fast path for edges inside the largest component
    st = giant_b.alloc(h, ((size_t)n + 31) / 32 * 4, s);
    if (st != MST_OK) return record(h, st);
    launch_giant_bits(E, m, 0x9e3779b97f4a7c15ULL, label, n, &h->ds->giant_root, giant_b.as<uint32_t>(), h->sms, s);
    a.giant_bits = giant_b.as<uint32_t>();
  }
  if (mode == CM_DEDUPE) {
    const uint64_t slots = next_pow2(2 * m < 1024 ? 1024 : 2 * m);
    st = table_b.alloc(h, slots * sizeof(HashSlot), s);
    if (st != MST_OK) return record(h, st);
    if (cudaMemsetAsync(table_b.p, 0xff, slots * sizeof(HashSlot), s) != cudaSuccess) return record_cuda(h, __LINE__);
    a.table = table_b.as<HashSlot>();
    a.tmask = slots - 1;
    launch_hash_insert(E, m, a.table, a.tmask, &h->ds->err, h->sms, s);
  }
  a.st = next_scan(h, CNT_USER);
  if (cudaMemsetAsync(&h->ds->count[CNT_USER], 0, sizeof(u64), s) != cudaSuccess) return record_cuda(h, __LINE__);
  launch_compact(mode, a, m, s);
  if (cudaMemcpyAsync(d_out_count, &h->ds->count[CNT_USER], 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return record_cuda(h, __LINE__);
  return record(h, readback(h, s));
}

mst_status mst_step_relabel(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                            const uint32_t *d_w, const uint32_t *d_id, const uint32_t *d_label, uint32_t *d_ou,
                            uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid, uint64_t *d_out_count, void *stream) {
  if (!d_label && m > 0) return MST_ERR_INVALID_ARG;
  return step_compact(h, CM_RELABEL, n, m, d_u, d_v, d_w, d_id, d_label, 0, d_ou, d_ov, d_ow, d_oid, d_out_count,
                      stream);
}

mst_status mst_step_dedupe(mst_handle h, uint64_t m, const uint32_t *d_u, const uint32_t *d_v, const uint32_t *d_w,
                           const uint32_t *d_id, uint32_t *d_ou, uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid,
                           uint64_t *d_out_count, void *stream) {
  if (!h || h->cfg.dedupe != MST_DEDUPE_SORT)
    return step_compact(h, CM_DEDUPE, 0, m, d_u, d_v, d_w, d_id, nullptr, 0, d_ou, d_ov, d_ow, d_oid, d_out_count,
                        stream);
  // sort variant: 32-bit ends, weights and ids, so the pair and (w, id) keys take 64 bits each
  if (!d_out_count || (m > 0 && (!d_u || !d_v || !d_w || !d_ou || !d_ov || !d_ow || !d_oid)))
    return record(h, MST_ERR_INVALID_ARG);
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (clear_device_flags(h, s) != MST_OK ||
      cudaMemsetAsync(&h->ds->count[CNT_USER], 0, sizeof(u64), s) != cudaSuccess)
    return record_cuda(h, __LINE__);
  Buf id_b, sd_b;
  mst_status st = MST_OK;
  const uint32_t *ids = d_id;
  if (m > 0 && !ids) {  // implicit ids: the index
    st = id_b.alloc(h, m * 4, s);
    if (st != MST_OK) return record(h, st);
    launch_iota(id_b.as<uint32_t>(), m, h->sms, s);
    ids = id_b.as<uint32_t>();
  }
  st = sd_b.alloc(h, sort_dedupe_scratch_bytes(m, h->sms), s);
  if (st != MST_OK) return record(h, st);
  CompactArgs cd{};
  cd.shape = shape_index(h->cfg.block_threads, h->cfg.items_per_thread);
  cd.in = EdgeList{d_u, d_v, d_w, ids};
  cd.m = m;
  cd.out = EdgeOut{d_ou, d_ov, d_ow, d_oid};
  cd.st = next_scan(h, CNT_USER);
  launch_sort_dedupe(cd.in, m, 32, 32, 32, cd, sd_b.p, h->sms, s);
  if (cudaMemcpyAsync(d_out_count, &h->ds->count[CNT_USER], 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return record_cuda(h, __LINE__);
  return record(h, readback(h, s));
}

mst_status mst_step_partition(mst_handle h, uint64_t m, const uint32_t *d_u, const uint32_t *d_v, const uint32_t *d_w,
                              const uint32_t *d_id, uint64_t pivot, uint32_t *d_ou, uint32_t *d_ov, uint32_t *d_ow,
                              uint32_t *d_oid, uint64_t *d_out_count, void *stream) {
  return step_compact(h, CM_PARTITION, 0, m, d_u, d_v, d_w, d_id, nullptr, pivot, d_ou, d_ov, d_ow, d_oid,
                      d_out_count, stream);
}

mst_status mst_step_filter(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_u, const uint32_t *d_v,
                           const uint32_t *d_w, const uint32_t *d_id, uint64_t pivot, uint32_t *d_P, uint32_t *d_ou,
                           uint32_t *d_ov, uint32_t *d_ow, uint32_t *d_oid, uint64_t *d_out_count, void *stream) {
  if (!h || !d_P) return MST_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    Solve S(h, s, n, 0);
    S.parent = d_P;
    if (clear_device_flags(h, s) != MST_OK) return record_cuda(h, __LINE__);
    launch_range_check(d_P, n, n, &h->ds->err, h->sms, s);  // P is walked: every entry must name a vertex
    mst_status st = readback(h, s);
    if (st != MST_OK) return record(h, st);
    st = S.compress_all();
    if (st != MST_OK) return record(h, st);
  }
  return step_compact(h, CM_FILTER, n, m, d_u, d_v, d_w, d_id, d_P, pivot, d_ou, d_ov, d_ow, d_oid, d_out_count,
                      stream);
}

mst_status mst_step_pivot(mst_handle h, uint64_t m, const uint32_t *d_w, const uint32_t *d_id, uint64_t state,
                          uint32_t sample, uint64_t *d_pivot, void *stream) {
  if (!h || !d_pivot || sample == 0 || (m > 0 && !d_w)) return MST_ERR_INVALID_ARG;
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  Buf sb;
  mst_status st = sb.alloc(h, (size_t)sample * 8, s);
  if (st != MST_OK) return record(h, st);
  const EdgeList E{nullptr, nullptr, d_w, d_id};
  if (!launch_pivot_coop(E, m, state, sample, sb.as<u64>(), h->pivot_scratch, (u64 *)d_pivot, s))
    launch_pivot(E, m, nullptr, state, sample, sb.as<u64>(), (u64 *)d_pivot, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return record_cuda(h, __LINE__);
  return record(h, MST_OK);
}

mst_status mst_step_tile_contract(mst_handle h, uint32_t n, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                                  const uint32_t *d_w, uint32_t tile_vertices, uint32_t *d_parent, uint32_t *d_chosen,
                                  void *stream) {
  if (!h || !d_parent || !d_chosen || (m > 0 && (!d_src || !d_dst || !d_w))) return MST_ERR_INVALID_ARG;
  if (tile_vertices < 32 || tile_vertices > 4096) return record(h, MST_ERR_INVALID_ARG);
  if (m >= (1ULL << 32)) return record(h, MST_ERR_TOO_LARGE);
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const mst_config saved = h->cfg;
  h->cfg.tile_contract = 1;
  h->cfg.tile_vertices = tile_vertices;
  h->cfg.tile_filter = 0;  // the step contracts exactly what the rounds without filtering contract
  mst_status st;
  {
    Solve S(h, s, n, m);
    st = S.init(d_parent, d_chosen);
    if (st == MST_OK) {
      S.src = d_src;
      S.dst = d_dst;
      S.w_in = d_w;
      ListBuf out;
      uint64_t mo = 0;
      bool applied = false;
      st = S.tile_preprocess(d_w, false, out, mo, applied);
      if (st == MST_OK && cudaStreamSynchronize(s) != cudaSuccess) st = MST_ERR_CUDA;
    }
  }
  h->cfg = saved;
  return record(h, st);
}

mst_status mst_step_finalize(mst_handle h, uint64_t m, const uint32_t *d_chosen, const uint32_t *d_w,
                             uint32_t *d_msf_ids, uint32_t *d_msf_count, uint64_t *d_total_weight, void *stream) {
  if (!h || !d_msf_count || !d_total_weight || (m > 0 && (!d_chosen || !d_w || !d_msf_ids)))
    return MST_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  mst_status st = ensure_status(h, (m + 31) / 32, s);
  if (st != MST_OK) return record(h, st);
  if (clear_device_flags(h, s) != MST_OK || cudaMemsetAsync(d_total_weight, 0, 8, s) != cudaSuccess)
    return record_cuda(h, __LINE__);
  launch_finalize(d_chosen, m, d_w, d_msf_ids, d_msf_count, (u64 *)d_total_weight, next_scan(h, CNT_AUX), s);
  return record(h, readback(h, s));
}

}  // extern "C"
