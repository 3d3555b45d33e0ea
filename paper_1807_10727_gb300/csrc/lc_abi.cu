// C ABI of liblc.so (include/lc.h): context management and the host-driven
// phase loop of LocalContraction (arXiv 1807.10727, Section 3), one CUDA
// stream, one device synchronisation per phase to read the phase's sizes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lc_internal.cuh"

using namespace lc;

namespace lc {

const char* kernel_name(int id) {
  static const char* names[] = {
      "init_keys",   "edge_min_soa", "edge_min_packed", "jump",          "relabel_soa",
      "relabel_packed", "relabel_split", "sort_hist", "hist_scan",     "sort_pass",
      "scan_flags",
      "unique_rename", "propagate",  "bucket_bounds",   "bucket_dedup",  "rename",
      "unmix",         "batch",      "two_hop",         "open_min",      "tree_names",
      "union_find",    "m2l_group",  "m2l_select",      "m2l_hop",       "m2l_target",
      "identity",      "rank_probe", "filter_hll",   "bucket_edges",  "seg_dedup"};
  static_assert(sizeof(names) / sizeof(names[0]) == kNumKernels, "one name per kernel");
  return (id >= 0 && id < kNumKernels) ? names[id] : "unknown";
}

cudaEvent_t Prof::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Prof::resolve() {
  for (auto& t : pending) {
    float ms_ = 0.f;
    if (cudaEventElapsedTime(&ms_, std::get<1>(t), std::get<2>(t)) == cudaSuccess)
      ms[std::get<0>(t)] += ms_;
    pool.push_back(std::get<1>(t));
    pool.push_back(std::get<2>(t));
  }
  pending.clear();
}

void Prof::reset() {
  for (int k = 0; k < kNumKernels; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
}

void Prof::release() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

}  // namespace lc

namespace {

// Level storage of one phase: the root map, the min-original-id of each
// node, and the keep ranks of the nodes (see rank_words).
struct Level {
  uint32_t n;
  uint32_t* root;
  uint32_t* mo;
  uint64_t* rank;  // keep ranks, rank_words(n) words
};

// Test hook: the allocation with this number (counted from the last
// lc_fail_alloc call) fails; 0 = off.
std::atomic<uint64_t> g_fail_at{0};
std::atomic<uint64_t> g_alloc_no{0};

bool injected_failure() {
  if (g_fail_at.load() == 0) return false;
  const uint64_t no = g_alloc_no.fetch_add(1) + 1;
  uint64_t at = no;
  return g_fail_at.compare_exchange_strong(at, 0);  // one shot
}

// Where a context's device memory comes from: cudaMalloc, or (contexts of a
// server) stream-ordered allocation from the server's memory pool, which
// neither allocation nor release synchronises with the device.
struct MemSource {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;  // pool allocations and releases are ordered here
};

template <class T>
cudaError_t dev_alloc(const MemSource& ms, T** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  void* q = nullptr;
  const cudaError_t e = ms.pool ? cudaMallocFromPoolAsync(&q, bytes, ms.pool, ms.stream)
                                : cudaMalloc(&q, bytes);
  if (e == cudaSuccess) *p = static_cast<T*>(q);
  return e;
}

void dev_free(const MemSource& ms, const void* p) {
  if (p == nullptr) return;
  if (ms.pool) cudaFreeAsync(const_cast<void*>(p), ms.stream);
  else cudaFree(const_cast<void*>(p));
}

template <class T>
cudaError_t host_alloc(T** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  void* q = nullptr;
  const cudaError_t e = cudaMallocHost(&q, bytes);
  if (e == cudaSuccess) *p = static_cast<T*>(q);
  return e;
}

// Bump arena for the per-phase arrays; grows by whole chunks when a run needs
// more than the first chunk (only when the phases shrink slowly).
struct Arena {
  std::vector<std::pair<uint32_t*, uint64_t>> chunks;  // (base, words)
  size_t cur = 0;
  uint64_t used = 0;
  bool fixed = false;  // never grow: running out is an allocation failure
  const MemSource* ms = nullptr;
  cudaError_t init(uint64_t words) {
    uint32_t* p = nullptr;
    cudaError_t e = dev_alloc(*ms, &p, std::max<uint64_t>(words, 1024) * 4);
    if (e != cudaSuccess) return e;
    chunks.push_back({p, std::max<uint64_t>(words, 1024)});
    return cudaSuccess;
  }
  void reset() { cur = 0; used = 0; }
  uint32_t* alloc(uint64_t words, cudaError_t* err) {
    words = (words + 63) & ~63ull;  // 256-byte aligned pieces
    if (fixed && injected_failure()) {  // a fixed arena's pieces count for the test hook
      *err = cudaErrorMemoryAllocation;
      return nullptr;
    }
    while (cur < chunks.size()) {
      if (used + words <= chunks[cur].second) {
        uint32_t* p = chunks[cur].first + used;
        used += words;
        return p;
      }
      ++cur;
      used = 0;
    }
    if (fixed) {
      *err = cudaErrorMemoryAllocation;
      return nullptr;
    }
    uint64_t sz = std::max<uint64_t>(words, chunks.empty() ? words : chunks.back().second);
    uint32_t* p = nullptr;
    *err = dev_alloc(*ms, &p, sz * 4);
    if (*err != cudaSuccess) return nullptr;
    chunks.push_back({p, sz});
    cur = chunks.size() - 1;
    used = words;
    return p;
  }
  void release() {
    for (auto& c : chunks) dev_free(*ms, c.first);
    chunks.clear();
  }
};

uint64_t host_mix(uint64_t z) { return splitmix_mix(z); }

// Phases with at least this many edges use the relabel's device-wide
// duplicate cache, and size their deduplication buckets from a HyperLogLog
// estimate of the distinct keys read back after the relabel (below it the
// block caches and the dedup are cheap, and a mid-phase wait would cost more
// than it saves).
constexpr uint64_t kGCacheMinEdges = 1ull << 22;
constexpr uint32_t kGCacheSlots = 1u << 23;  // default size (64 MB)
constexpr int kGCacheAdmit = 3;              // default admission: 1 in 8 occurrences

// Stream seed of phase i: output i+1 of the SplitMix64 stream seeded with seed.
uint64_t phase_seed(uint64_t seed, uint32_t i) { return host_mix(seed + (uint64_t)(i + 1) * kGamma); }

int bits_for(uint32_t n) {
  int b = 1;
  while (b < 32 && (1ull << b) < n) ++b;
  return b;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

// Progress of one run of the phase loop (see run_begin / run_complete).
struct RunState {
  enum State { kDone = 0, kRelabel, kPhase, kSortPhase, kLabels } state = kDone;
  lc_status st = LC_OK;
  bool merge_step = false;  // the level in flight is phase i's MergeToLarge step
  uint32_t passes = 0;      // partition passes planned for the level in flight
  bool filtered = false;    // the level's keys went through the filter pass
  bool seg = false;         // the kept keys lie in segment regions (segmented dedup)
  bool pre0 = false;        // phase 0's ranks, bucket counts and minimum ran as the input
                            // arrived (lc_run_host)
  uint32_t pre0_chunks = 0; // > 0: each of these input chunks was grouped on arrival
  uint32_t* d_labels = nullptr;
  uint32_t i = 0, ni = 0;
  uint64_t mi = 0;
  const uint64_t* packed = nullptr;  // current edges when not the input
  uint32_t* mo_cur = nullptr;
  Level lv{};
  uint32_t* mo_next = nullptr;
  int bits = 1;
  uint64_t *keys = nullptr, *alt = nullptr, *part = nullptr, *next = nullptr;
  std::vector<uint64_t> hn, hm;
};

// A batch of independent graphs run as one (see BatchKeys in lc_round.cu).
struct BatchState {
  uint32_t k = 0;
  uint64_t* d_seeds = nullptr;  // [k] rank seeds
  uint32_t* d_voff0 = nullptr;  // [k+1] vertex offsets of the input
  uint64_t* d_eoff = nullptr;   // [k+1] edge offsets of the input
  uint64_t* d_rk = nullptr;     // [k] phase seeds of the current phase (BatchView::gs)
  uint32_t* d_gid = nullptr;    // [n] graph of every vertex of the current level
  const uint32_t* user_src = nullptr;  // caller's edges, local ids
  const uint32_t* user_dst = nullptr;
  std::vector<uint64_t> h_eoff;
  std::vector<uint32_t> h_voff0;
  std::vector<uint32_t*> voff;  // per level: [k+1] offsets (level 0: d_voff0)
  std::vector<uint32_t*> mcnt;  // per level i >= 1: [k] edges per graph
};

struct lc_ctx {
  uint32_t n = 0;
  uint64_t m = 0;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  MemSource mem;                // device memory source (stream follows `stream`)
  unsigned char* pinned = nullptr;  // borrowed pinned block for h_ctr / h_hll (servers)
  Launch L{};
  Prof prof;
  lc_variant variant = LC_VARIANT_FOREST;
  uint64_t finish_edges = 0;
  cudaStream_t copy_stream = nullptr;  // lc_run_host: input copies, chunk by chunk
  cudaEvent_t copy_ev = nullptr;       // lc_run_host: the last chunk copied
  uint64_t host_chunk_edges = 1ull << 25;
  std::vector<uint32_t> merge_alpha;  // MergeToLarge parameter of phase i (0: off)

  const uint32_t* src = nullptr;
  const uint32_t* dst = nullptr;
  uint32_t* own_src = nullptr;
  uint32_t* own_dst = nullptr;
  uint32_t* own_labels = nullptr;

  unsigned long long* minkey = nullptr;
  unsigned long long* minkey2 = nullptr;  // second-hop minima (two-hop variant only)
  unsigned long long* gcache = nullptr;   // relabel's device-wide duplicate cache
  uint32_t gcache_slots = 0;
  int gcache_admit = kGCacheAdmit;        // log2 of the cache's admission period
  uint32_t* d_hll = nullptr;              // HyperLogLog registers of the relabel's keys
  uint32_t* h_hll = nullptr;              // (pinned host copy)
  uint32_t* flags = nullptr;  // bitmap, flag_words(n) words
  uint64_t* ebuf[2] = {nullptr, nullptr};
  Counters* ctr = nullptr;
  Counters* h_ctr = nullptr;
  SortScratch sort;
  Arena arena;
  std::vector<Level> levels;

  uint32_t* bounds = nullptr;  // bucket boundaries of the hashed dedup
  uint64_t fallbacks = 0;      // phases that needed the full-sort dedup
  bool dedup_sort = false;     // deduplicate by a full radix sort every phase
  uint64_t window_bytes = 192ull << 20;  // L2 budget of one phase-0 minimum pass
  uint64_t relabel_window_bytes = 160ull << 20;  // root-array size above which relabel splits
  uint32_t* bucket_scratch = nullptr;            // counts and fill counters of the edge buckets
  uint32_t* chunk_scratch = nullptr;             // lc_run_host: bucket scratch per input chunk
  uint64_t chunk_scratch_bytes = 0;
  uint64_t* chunk_tile_buf = nullptr;            // lc_run_host: relabel tiles over the chunks
  uint64_t chunk_tile_bytes = 0;
  uint32_t bucket_blocks = 0;                    // phase-0 edge buckets: 0 auto, 1 off, else blocks
  uint64_t bucket_window_bytes = 64ull << 20;    // auto: two blocks of minima fit in this
  uint32_t bucket_min_vertices = 1u << 23;       // auto: bucket only graphs of this many vertices
  uint64_t* dtable = nullptr;                    // slices of the segmented deduplication
  uint64_t dtable_slots = 0;
  uint64_t table_cap = 0;                        // slots the segmented dedup may use (0: all)
  bool seg_dedup = true;                         // large phases deduplicate by table slices
  uint32_t target_permille = 1000;               // scale of the distinct-key estimate (tests)
  uint64_t late_min_edges = 1ull << 22;          // phases this large plan their dedup late
  bool cache_in_relabel = false;                 // segmented phases probe the cache in the relabel
  uint32_t jump_bits_min_vertices = 1u << 23;    // sparse phases this large chase with a root bitmap

  uint32_t max_rounds = 0;  // phase cap (0: 64 + 4 log2 n)
  uint32_t last_rounds = 0;
  std::vector<uint64_t> last_mp;
  std::vector<uint64_t> last_emitted;
  std::vector<uint32_t> last_passes;  // partition passes of each phase's hashed dedup
  std::vector<uint64_t> last_kept;    // keys each phase deduplicated

  cudaEvent_t ev = nullptr;  // completion of the work enqueued last (none: sync the stream)
  RunState rs;
  BatchState* batch = nullptr;
  uint64_t tag = 0;    // last value stamped into the device counters
  uint32_t n_cap = 0;  // sizes the buffers were allocated for (a context may be
  uint64_t m_cap = 0;  // re-bound to any smaller graph, see ctx_rebind)
};

#define LC_TRY(call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return status_of(e_);      \
  } while (0)

static lc_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return LC_OK;
  if (e == cudaErrorMemoryAllocation) return LC_ERR_OOM;
  return LC_ERR_CUDA;
}

static void free_ctx(lc_ctx* c) {
  if (!c) return;
  dev_free(c->mem, c->own_src);
  dev_free(c->mem, c->own_dst);
  dev_free(c->mem, c->own_labels);
  dev_free(c->mem, c->minkey);
  dev_free(c->mem, c->minkey2);
  dev_free(c->mem, c->gcache);
  dev_free(c->mem, c->d_hll);
  if (c->h_hll && !c->pinned) cudaFreeHost(c->h_hll);
  dev_free(c->mem, c->flags);
  dev_free(c->mem, c->ebuf[0]);
  dev_free(c->mem, c->ebuf[1]);
  dev_free(c->mem, c->ctr);
  if (c->h_ctr && !c->pinned) cudaFreeHost(c->h_ctr);
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->copy_ev) cudaEventDestroy(c->copy_ev);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->batch) {
    dev_free(c->mem, c->batch->d_seeds);
    dev_free(c->mem, c->batch->d_voff0);
    dev_free(c->mem, c->batch->d_eoff);
    dev_free(c->mem, c->batch->d_rk);
    dev_free(c->mem, c->batch->d_gid);
    delete c->batch;
  }
  dev_free(c->mem, c->sort.status);
  dev_free(c->mem, c->sort.hist);
  dev_free(c->mem, c->sort.tickets);
  dev_free(c->mem, c->bounds);
  dev_free(c->mem, c->bucket_scratch);
  dev_free(c->mem, c->chunk_scratch);
  dev_free(c->mem, c->chunk_tile_buf);
  dev_free(c->mem, c->dtable);
  c->arena.release();
  c->prof.release();
  delete c;
}

// Slots of the segmented-deduplication table for up to m keys: twice m,
// rounded up to a power of two, at least kSegs * 64, at most 2^28 (2 GB).
static uint64_t table_slots_for(uint64_t m) {
  uint64_t t = (uint64_t)kSegs * 64;
  while (t < 2 * m && t < (1ull << 28)) t <<= 1;
  return t;
}

// Buffers of the phases that plan their deduplication after the relabel:
// the device-wide duplicate cache, the HyperLogLog registers (and their
// pinned host copy) and the segmented-deduplication table.
static cudaError_t alloc_late(lc_ctx* c) {
  cudaError_t e = cudaSuccess;
  if (c->gcache == nullptr) {
    c->gcache_slots = kGCacheSlots;
    e = dev_alloc(c->mem, &c->gcache, 8ull * c->gcache_slots);
    if (e != cudaSuccess) {
      c->gcache_slots = 0;
      return e;
    }
  }
  if (c->d_hll == nullptr && (e = dev_alloc(c->mem, &c->d_hll, 4ull * kHllRegs)) != cudaSuccess) return e;
  if (c->h_hll == nullptr) {
    if (c->pinned) c->h_hll = reinterpret_cast<uint32_t*>(c->pinned + 256);
    else if ((e = host_alloc(&c->h_hll, 4ull * kHllRegs)) != cudaSuccess) return e;
  }
  if (c->dtable == nullptr) {
    const uint64_t slots = table_slots_for(c->m_cap);
    if ((e = dev_alloc(c->mem, &c->dtable, 8ull * slots)) != cudaSuccess) return e;
    c->dtable_slots = slots;
  }
  return cudaSuccess;
}

static lc_status alloc_ctx(lc_ctx* c) {
  const uint64_t n = c->n, m = c->m;
  c->n_cap = c->n;
  c->m_cap = c->m;
  LC_TRY(dev_alloc(c->mem, &c->minkey, std::max<uint64_t>(n, 1) * 8));
  LC_TRY(dev_alloc(c->mem, &c->flags, 4 * (flag_words(n) + 4)));
  LC_TRY(dev_alloc(c->mem, &c->ebuf[0], std::max<uint64_t>(m, 2) * 8));
  LC_TRY(dev_alloc(c->mem, &c->ebuf[1], std::max<uint64_t>(m, 2) * 8));
  LC_TRY(dev_alloc(c->mem, &c->ctr, sizeof(Counters)));
  // initialisation is ordered on the context's stream, and lc_create waits
  // for it, so the context may then be used from any stream
  LC_TRY(cudaMemsetAsync(c->ctr, 0, sizeof(Counters), c->stream));
  if (c->pinned) c->h_ctr = reinterpret_cast<Counters*>(c->pinned);
  else LC_TRY(host_alloc(&c->h_ctr, sizeof(Counters)));
  LC_TRY(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
  c->sort.status_words = std::max(sort_status_words(m), sort_status_words(n));
  LC_TRY(dev_alloc(c->mem, &c->sort.status, c->sort.status_words * 8));
  LC_TRY(cudaMemsetAsync(c->sort.status, 0, c->sort.status_words * 8, c->stream));
  LC_TRY(dev_alloc(c->mem, &c->sort.hist, sizeof(uint32_t) * kMaxPasses * kRadixMax));
  LC_TRY(dev_alloc(c->mem, &c->sort.tickets, sizeof(unsigned) * 16));
  LC_TRY(dev_alloc(c->mem, &c->bounds, sizeof(uint32_t) * ((1ull << hash_bits_for(m)) + 1)));
  LC_TRY(dev_alloc(c->mem, &c->bucket_scratch, sizeof(uint32_t) * kBucketScratchWords));
  if (m >= kGCacheMinEdges) LC_TRY(alloc_late(c));
  // first arena chunk: 3 arrays per level for levels whose sizes sum to 2n,
  // plus the next level's min-original-id array
  LC_TRY(c->arena.init(4 * (2 * n + 256)));
  return LC_OK;
}

// lc_create with a choice of memory source: `pool` non-null allocates the
// context's device memory stream-ordered from that pool on `stream`, and
// `pinned` (kPinnedBlock bytes) holds its host counters instead of its own
// pinned allocation (both for the contexts of a server).
constexpr size_t kPinnedBlock = 256 + 4 * kHllRegs;

static lc_status create_ctx(uint32_t n, const uint32_t* d_src, const uint32_t* d_dst, uint64_t m,
                            uint64_t seed, cudaStream_t stream, cudaMemPool_t pool,
                            unsigned char* pinned, lc_ctx** out) {
  if (out == nullptr) return LC_ERR_INVALID;
  *out = nullptr;
  if ((d_src == nullptr) != (d_dst == nullptr)) return LC_ERR_INVALID;
  if (m > 0xFFFFFFFFull) return LC_ERR_INVALID;
  if (n == 0 && m > 0) return LC_ERR_INVALID;
  lc_ctx* c = new (std::nothrow) lc_ctx();
  if (!c) return LC_ERR_OOM;
  c->n = n;
  c->m = m;
  c->seed = seed;
  c->stream = stream;
  c->mem = MemSource{pool, stream};
  c->pinned = pinned;
  c->arena.ms = &c->mem;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return LC_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(&c->L.sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return LC_ERR_CUDA;
  }
  c->L.stream = c->stream;
  c->L.prof = &c->prof;
  c->src = d_src;
  c->dst = d_dst;
  lc_status st = alloc_ctx(c);
  if (st == LC_OK && d_src == nullptr) {
    cudaError_t e = dev_alloc(c->mem, &c->own_src, std::max<uint64_t>(m, 1) * 4);
    if (e == cudaSuccess) e = dev_alloc(c->mem, &c->own_dst, std::max<uint64_t>(m, 1) * 4);
    if (e == cudaSuccess) e = dev_alloc(c->mem, &c->own_labels, std::max<uint64_t>(n, 1) * 4);
    st = status_of(e);
    c->src = c->own_src;
    c->dst = c->own_dst;
  }
  if (st == LC_OK) st = status_of(cudaStreamSynchronize(c->stream));
  if (st != LC_OK) {
    free_ctx(c);
    if (pool) cudaStreamSynchronize(stream);  // the releases are ordered there
    cudaGetLastError();
    return st;
  }
  *out = c;
  return LC_OK;
}

extern "C" lc_status lc_create(uint32_t n, const uint32_t* d_src, const uint32_t* d_dst,
                               uint64_t m, uint64_t seed, void* stream, lc_ctx** out) {
  return create_ctx(n, d_src, d_dst, m, seed, (cudaStream_t)stream, nullptr, nullptr, out);
}

extern "C" lc_status lc_fail_alloc(uint64_t k) {
  g_alloc_no.store(0);
  g_fail_at.store(k);
  return LC_OK;
}

extern "C" lc_status lc_configure(lc_ctx* c, lc_variant variant, uint64_t finish_edges) {
  if (!c) return LC_ERR_INVALID;
  if (variant != LC_VARIANT_FOREST && variant != LC_VARIANT_TWO_HOP && variant != LC_VARIANT_TREE)
    return LC_ERR_INVALID;
  // the finish threshold compares one graph's edge count; a batch has many
  if (finish_edges != 0 && c->batch != nullptr) return LC_ERR_INVALID;
  if (c->rs.state != RunState::kDone) return LC_ERR_INVALID;
  if (variant == LC_VARIANT_TWO_HOP && c->minkey2 == nullptr)
    LC_TRY(dev_alloc(c->mem, &c->minkey2, std::max<uint64_t>(c->n_cap, 1) * 8));
  c->variant = variant;
  c->finish_edges = finish_edges;
  return LC_OK;
}

extern "C" lc_status lc_set_merge_to_large(lc_ctx* c, const uint32_t* alpha, uint32_t count) {
  if (!c || (count > 0 && alpha == nullptr)) return LC_ERR_INVALID;
  if (count > 0 && c->batch != nullptr) return LC_ERR_INVALID;
  if (c->rs.state != RunState::kDone) return LC_ERR_INVALID;
  c->merge_alpha.assign(alpha, alpha + count);
  return LC_OK;
}

static uint32_t round_cap(uint32_t n) { return 64 + 4 * (uint32_t)bits_for(std::max(n, 2u)); }

// ---------------------------------------------------------------------------
// The phase loop as a state machine, so that one host thread can drive many
// contexts: run_begin enqueues phase 0, and each time the work enqueued last
// has completed (run_wait, or an event query), run_complete reads the phase's
// counters and enqueues the next phase, the dedup fallback, or the final label
// composition.

static lc_status record(lc_ctx* c) {
  LC_TRY(cudaGetLastError());
  if (c->ev) LC_TRY(cudaEventRecord(c->ev, c->stream));
  return LC_OK;
}

static lc_status enqueue_sort_dedup(lc_ctx* c);

// Device count of the keys the level in flight deduplicates.
static unsigned long long* kept_count(lc_ctx* c) {
  return c->rs.filtered ? &c->ctr->filtered : &c->ctr->emitted;
}

static lc_status enqueue_dedup(lc_ctx* c, const PassPlan& hplan, int hb, bool hist_ready);

static lc_status fail(lc_ctx* c, lc_status st) {
  c->rs.st = st;
  c->rs.state = RunState::kDone;
  return st;
}

// Vertex blocks of the phase-0 edge buckets for a graph of n vertices (1: the
// input edges are read as given).
static uint32_t bucket_blocks(const lc_ctx* c, uint32_t n) {
  if (c->bucket_scratch == nullptr || c->bucket_blocks == 1) return 1;
  if (c->bucket_blocks > 1) return std::min(c->bucket_blocks, std::max(n, 2u));
  if (n < c->bucket_min_vertices) return 1;
  return bucket_blocks_for(n, c->bucket_window_bytes);
}

// Enqueue phase rs.i on (rs.ni, rs.mi): steps (a)-(d) and the copy of the
// phase counters to the host.
static lc_status enqueue_phase(lc_ctx* c) {
  RunState& r = c->rs;
  const Launch& L = c->L;
  cudaError_t aerr = cudaSuccess;
  const uint32_t i = r.i, ni = r.ni;
  const uint64_t mi = r.mi;
  r.lv = Level{ni, c->arena.alloc(ni, &aerr), r.mo_cur, nullptr};
  if (aerr != cudaSuccess) return fail(c, status_of(aerr));
  r.lv.rank = reinterpret_cast<uint64_t*>(c->arena.alloc(2 * rank_words(ni), &aerr));
  if (aerr != cudaSuccess) return fail(c, status_of(aerr));
  r.mo_next = c->arena.alloc(ni, &aerr);
  if (aerr != cudaSuccess) return fail(c, status_of(aerr));
  const uint64_t rk = phase_seed(c->seed, i);
  r.bits = bits_for(ni);
  unsigned* err = &c->ctr->err;
  BatchView bv{};
  if (BatchState* b = c->batch) {
    if (i > 0) {
      // per-graph offsets and edge counts of this level, from the last level
      uint32_t* voff = c->arena.alloc(b->k + 1, &aerr);
      if (aerr != cudaSuccess) return fail(c, status_of(aerr));
      uint32_t* mcnt = c->arena.alloc(b->k, &aerr);
      if (aerr != cudaSuccess) return fail(c, status_of(aerr));
      batch_next_level(b->voff.back(), c->levels.back().rank, b->k, voff, r.packed, mi, mcnt, ni,
                       b->d_gid, L);
      b->voff.push_back(voff);
      b->mcnt.push_back(mcnt);
    }
    batch_phase_seeds(b->d_seeds, b->k, i, b->voff.back(), b->d_rk, L);
    bv = BatchView{b->d_rk, b->voff.back(), b->k, b->d_gid};
  }
  const BatchView* bp = c->batch ? &bv : nullptr;
  // the input edges are read only by phase 0 itself (a merge step after
  // phase 0 works on the packed edges that phase 0 wrote)
  const bool first = i == 0 && !r.merge_step;
  const uint32_t* src0 = first ? c->src : nullptr;
  const uint32_t* dst0 = first ? c->dst : nullptr;
  // current edges in packed form (phases >= 1, or phase 0's bucketed input)
  const uint64_t* pk = r.packed;
  const uint32_t nb = first ? bucket_blocks(c, ni) : 1u;
  const uint64_t* tiles = nullptr;  // relabel tile list (chunk-local grouping)
  const unsigned long long* d_ntiles = nullptr;
  if (nb > 1 && mi > 0) {
    // phase 0: group the input edges by vertex-block pair, so that the steps
    // below gather from an L2-sized slice of the per-vertex arrays at a time;
    // the grouped copy goes to the buffer the relabel does not write
    uint64_t* grouped = c->ebuf[1];
    if (r.pre0 && r.pre0_chunks > 0) {
      // grouped chunk by chunk as the input arrived: the relabel takes the
      // (bucket, chunk) runs through a tile list, in bucket order
      chunk_tiles(c->chunk_scratch, r.pre0_chunks, std::max<uint64_t>(c->host_chunk_edges, 1),
                  mi, ni, nb, kRelabelTileEdges, c->chunk_tile_buf + 2,
                  reinterpret_cast<unsigned long long*>(c->chunk_tile_buf), err, L);
      tiles = c->chunk_tile_buf + 2;
      d_ntiles = reinterpret_cast<const unsigned long long*>(c->chunk_tile_buf);
    } else if (r.pre0)
      bucket_place(src0, dst0, mi, ni, nb, grouped, c->bucket_scratch, err, L);
    else
      bucket_edges(src0, dst0, mi, ni, nb, grouped, c->bucket_scratch, err, L);
    src0 = dst0 = nullptr;
    pk = grouped;
  }
  if (r.merge_step) {
    // MergeToLarge on the graph that phase i just produced
    const Level& prev = c->levels.back();
    MergeScratch ms{};
    uint32_t** u32s[] = {&ms.cnt, &ms.off, &ms.fill, &ms.list};
    for (uint32_t** q : u32s) {
      *q = c->arena.alloc(ni, &aerr);
      if (aerr != cudaSuccess) return fail(c, status_of(aerr));
    }
    ms.members = c->arena.alloc(prev.n, &aerr);
    if (aerr != cudaSuccess) return fail(c, status_of(aerr));
    ms.cand = reinterpret_cast<unsigned long long*>(c->arena.alloc(2ull * prev.n, &aerr));
    if (aerr != cudaSuccess) return fail(c, status_of(aerr));
    unsigned long long** u64s[] = {&ms.prio, &ms.h1, &ms.h2};
    for (unsigned long long** q : u64s) {
      *q = reinterpret_cast<unsigned long long*>(c->arena.alloc(2ull * ni, &aerr));
      if (aerr != cudaSuccess) return fail(c, status_of(aerr));
    }
    ms.ctrs = c->arena.alloc(3, &aerr);
    if (aerr != cudaSuccess) return fail(c, status_of(aerr));
    ms.big = c->arena.alloc(merge_big_words(prev.n), &aerr);
    if (aerr != cudaSuccess) return fail(c, status_of(aerr));
    merge_to_large_names(prev.root, prev.rank, prev.n, rk, c->merge_alpha[i], r.packed, mi, ni,
                         r.lv.root, r.lv.mo, ms, err, L);
  } else if (first && r.pre0) {
    // (a) ran with the input copy; each vertex's min original id = itself
    identity_labels(r.lv.mo, ni, L);
  } else {
    // (a): ranks (and, in phase 0, each vertex's min original id = itself)
    init_keys(c->minkey, first ? r.lv.mo : nullptr, ni, rk, bp, L);
  }
  if (r.merge_step) {
    // names computed above
  } else if (c->finish_edges != 0 && mi <= c->finish_edges) {
    // small-graph finish: one node per connected component of G_i
    union_find_names(src0, dst0, pk, mi, ni, reinterpret_cast<uint32_t*>(c->minkey),
                     r.lv.root, r.lv.mo, err, L);
  } else if (c->variant == LC_VARIANT_TREE) {
    // (b) + (c): open-neighbourhood parent, names from the terminal 2-cycles
    if (cudaMemsetAsync(c->minkey, 0xFF, sizeof(unsigned long long) * ni, c->stream) !=
        cudaSuccess)
      return fail(c, LC_ERR_CUDA);
    edge_min(src0, dst0, pk, mi, ni, rk, c->minkey, err, c->window_bytes, bp, L, true);
    tree_names(c->minkey, r.lv.root, r.lv.mo, ni, rk, bp, err, L);
  } else {
    // (b): closed-neighbourhood minimum (phase 0 of lc_run_host: done as the
    // input arrived)
    if (!(first && r.pre0))
      edge_min(src0, dst0, pk, mi, ni, rk, c->minkey, err, c->window_bytes, bp, L);
    if (c->variant == LC_VARIANT_TWO_HOP) {
      // second hop; names are label vertices, node minima in their own array
      uint32_t* nmo = c->arena.alloc(ni, &aerr);
      if (aerr != cudaSuccess) return fail(c, status_of(aerr));
      uint32_t* fpar = c->arena.alloc(ni, &aerr);
      if (aerr != cudaSuccess) return fail(c, status_of(aerr));
      two_hop_names(src0, dst0, pk, mi, ni, rk, bp, c->minkey, c->minkey2, fpar, r.lv.root,
                    r.lv.mo, nmo, err, L);
      r.lv.mo = nmo;
    } else {
      // (c): roots of the parent arborescences
      // (the node-flag bitmap, cleared below, holds the root bitmap meanwhile)
      jump(c->minkey, r.lv.root, r.lv.mo, ni, mi, c->flags, c->jump_bits_min_vertices, err, L);
    }
  }
  // (d): relabel, drop loops, deduplicate, compact
  if (cudaMemsetAsync(c->ctr, 0, 4 * sizeof(unsigned long long), c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->flags, 0, 4 * flag_words(ni), c->stream) != cudaSuccess)
    return fail(c, LC_ERR_CUDA);
  r.keys = (r.packed == c->ebuf[0]) ? c->ebuf[1] : c->ebuf[0];
  r.alt = (r.keys == c->ebuf[0]) ? c->ebuf[1] : c->ebuf[0];
  r.filtered = false;
  r.seg = false;
  const bool big = mi >= c->late_min_edges;
  // large phases plan their deduplication after the relabel, from the
  // estimated number of distinct keys; the others from m_i, with the
  // partition histogram fused into the relabel
  const bool late = !c->dedup_sort && big && c->d_hll != nullptr;
  // large phases with a table deduplicate by segments: the relabel counts
  // its keys per segment (the top kSegBits bits of the mixed key)
  const bool seg = late && c->seg_dedup && c->dtable != nullptr;
  PassPlan hplan{};
  const int hb = late ? 0 : hash_plan(mi, &hplan);
  if (!c->dedup_sort && !late) hist_reset(c->sort, L);
  PassPlan splan{};
  if (seg) {
    splan.passes = 1;
    splan.shift[0] = 64 - kSegBits;
    splan.bits[0] = kSegBits;
    if (cudaMemsetAsync(c->bucket_scratch, 0, sizeof(uint32_t) * kSegs, c->stream) != cudaSuccess)
      return fail(c, LC_ERR_CUDA);
  }
  if (late && cudaMemsetAsync(c->d_hll, 0, 4ull * kHllRegs, c->stream) != cudaSuccess)
    return fail(c, LC_ERR_CUDA);
  // the device-wide duplicate cache: in the relabel itself with the full
  // sort, else in the filter pass of a late-planned phase
  const bool use_gcache = c->gcache != nullptr && big;
  if (use_gcache &&
      cudaMemsetAsync(c->gcache, 0xFF, 8ull * c->gcache_slots, c->stream) != cudaSuccess)
    return fail(c, LC_ERR_CUDA);
  const bool gcache_in_relabel = use_gcache && (!late || (seg && c->cache_in_relabel));
  relabel(src0, dst0, pk, mi, ni, r.lv.root,
          r.bits, r.keys, &c->ctr->mprime, &c->ctr->emitted, !c->dedup_sort,
          seg ? &splan : (c->dedup_sort || late) ? nullptr : &hplan,
          seg ? c->bucket_scratch : c->sort.hist,
          (first && pk == nullptr) ? r.alt : nullptr,
          c->relabel_window_bytes, gcache_in_relabel ? c->gcache : nullptr,
          gcache_in_relabel ? c->gcache_slots : 0, c->gcache_admit, c->sort.tickets + 13, err, L,
          tiles, d_ntiles);
  if (late) {
    // drop repeats through the device-wide cache while sketching the distinct
    // count; the kept keys (counted in `filtered`) replace the relabelled ones
    if (cudaMemsetAsync(&c->ctr->filtered, 0, sizeof(unsigned long long), c->stream) !=
        cudaSuccess)
      return fail(c, LC_ERR_CUDA);
    if (seg) {
      // kept keys go straight to their segment's region
      seg_begin(c->bucket_scratch, L);
      const bool fcache = use_gcache && !gcache_in_relabel;
      filter_seg(r.keys, &c->ctr->emitted, mi, r.alt, &c->ctr->filtered,
                 fcache ? c->gcache : nullptr, fcache ? c->gcache_slots : 0,
                 c->gcache_admit, c->d_hll, c->bucket_scratch, err, L);
    } else {
      filter_hll(r.keys, &c->ctr->emitted, mi, r.alt, &c->ctr->filtered,
                 use_gcache ? c->gcache : nullptr, use_gcache ? c->gcache_slots : 0,
                 c->gcache_admit, c->d_hll, L);
    }
    std::swap(r.keys, r.alt);
    r.filtered = true;
    r.seg = seg;
    stamp_counters(c->ctr, ++c->tag, L);
    if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->h_hll, c->d_hll, 4ull * kHllRegs, cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
      return fail(c, LC_ERR_CUDA);
    r.state = RunState::kRelabel;
    lc_status st = record(c);
    return st == LC_OK ? st : fail(c, st);
  }
  return enqueue_dedup(c, hplan, hb, true);
}

// HyperLogLog estimate of the number of distinct keys from the registers
// (Flajolet, Fusy, Gandouet, Meunier 2007; linear counting for small counts).
static double hll_estimate(const uint32_t* reg) {
  const double m = kHllRegs;
  double sum = 0.0;
  uint32_t zeros = 0;
  for (int i = 0; i < kHllRegs; ++i) {
    sum += std::ldexp(1.0, -(int)reg[i]);
    zeros += reg[i] == 0 ? 1u : 0u;
  }
  double e = (0.7213 / (1.0 + 1.079 / m)) * m * m / sum;
  if (e <= 2.5 * m && zeros > 0) e = m * std::log(m / zeros);
  return e;
}

// Steps (d2) and (d3) of a segmented phase: the kept keys of segment s lie in
// its region of rs.keys; table slices of `slots` entries keep the distinct
// ones (into rs.alt).  Returns false, with the keys made contiguous again
// (rs.seg cleared), when the table cannot hold the slices.
static bool enqueue_seg_dedup(lc_ctx* c, uint64_t slots) {
  RunState& r = c->rs;
  const Launch& L = c->L;
  unsigned* err = &c->ctr->err;
  const uint64_t usable =
      c->table_cap ? std::min(c->table_cap, c->dtable_slots) : c->dtable_slots;
  if (!seg_dedup(r.keys, c->bucket_scratch, r.mi, c->dtable, usable, slots, r.alt,
                 &c->ctr->m_next, c->flags, r.ni, r.bits, c->sort.tickets + 11, err, L)) {
    seg_compact(r.keys, c->bucket_scratch, r.alt, L);
    std::swap(r.keys, r.alt);
    r.seg = false;
    return false;
  }
  r.passes = 0;
  r.part = r.keys;
  r.next = r.alt;
  scan_flags(c->flags, r.lv.rank, r.ni, r.lv.mo, r.mo_next, &c->ctr->n_next, c->sort, err, L);
  rename_edges(r.next, &c->ctr->m_next, r.mi, r.bits, r.lv.rank, r.ni, err, L);
  r.state = RunState::kPhase;
  stamp_counters(c->ctr, ++c->tag, L);
  if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    fail(c, LC_ERR_CUDA);
  else if (record(c) != LC_OK)
    fail(c, LC_ERR_CUDA);
  return true;
}

// Steps (d2) and (d3) of phase rs.i on the relabelled keys in rs.keys, then
// the copy of the phase counters to the host.
static lc_status enqueue_dedup(lc_ctx* c, const PassPlan& hplan, int hb, bool hist_ready) {
  RunState& r = c->rs;
  const Launch& L = c->L;
  unsigned* err = &c->ctr->err;
  const uint32_t ni = r.ni;
  const uint64_t mi = r.mi;
  r.passes = c->dedup_sort ? 0u : (uint32_t)hplan.passes;
  if (!c->dedup_sort) {
    int which = hash_dedup(r.keys, r.alt, kept_count(c), mi, hplan, hb, hist_ready, r.bits,
                           c->flags, ni, c->bounds, &c->ctr->m_next, c->sort, err, L);
    r.part = which ? r.alt : r.keys;
    r.next = which ? r.keys : r.alt;
    scan_flags(c->flags, r.lv.rank, ni, r.lv.mo, r.mo_next, &c->ctr->n_next, c->sort, err, L);
    rename_edges(r.next, &c->ctr->m_next, mi, r.bits, r.lv.rank, ni, err, L);
    r.state = RunState::kPhase;
  } else {
    r.part = r.keys;
    r.next = r.alt;
    r.state = RunState::kSortPhase;
    lc_status st = enqueue_sort_dedup(c);
    if (st != LC_OK) return st;
  }
  stamp_counters(c->ctr, ++c->tag, L);
  if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return fail(c, LC_ERR_CUDA);
  lc_status st = record(c);
  return st == LC_OK ? st : fail(c, st);
}

// Deduplicate the keys in rs.part by a full sort of all key bits, mark the
// endpoints of distinct keys, keep the first of each run renamed (output
// sorted, in rs.next).
static lc_status enqueue_sort_dedup(lc_ctx* c) {
  RunState& r = c->rs;
  const Launch& L = c->L;
  unsigned* err = &c->ctr->err;
  int w2 = radix_sort_u64(r.part, r.next, kept_count(c), r.mi, 2 * r.bits, c->sort, err,
                          c->flags, r.bits, L);
  uint64_t* sorted = w2 ? r.next : r.part;
  r.next = w2 ? r.part : r.next;
  scan_flags(c->flags, r.lv.rank, r.ni, r.lv.mo, r.mo_next, &c->ctr->n_next, c->sort, err, L);
  unique_rename(sorted, kept_count(c), r.mi, r.bits, r.lv.rank, r.ni, r.next,
                &c->ctr->m_next, c->sort, err, L);
  return LC_OK;
}

// (e): compose the phase maps top-down; level i's labels overwrite its root
// array in place (level 0 writes the caller's labels).
static lc_status enqueue_labels(lc_ctx* c) {
  const uint32_t R = (uint32_t)c->levels.size();
  for (int i = (int)R - 1; i >= 0; --i) {
    const Level& lv = c->levels[i];
    const uint32_t* up = (i + 1 < (int)R) ? c->levels[i + 1].root : nullptr;
    const uint32_t n_up = (i + 1 < (int)R) ? c->levels[i + 1].n : 0;
    uint32_t* out = i == 0 ? c->rs.d_labels : lv.root;
    propagate(lv.root, lv.rank, lv.mo, up, out, lv.n, n_up, &c->ctr->err, c->L);
  }
  if (c->batch) batch_localize(c->rs.d_labels, c->n, c->batch->d_voff0, c->batch->k, c->L);
  stamp_counters(c->ctr, ++c->tag, c->L);
  if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return fail(c, LC_ERR_CUDA);
  c->rs.state = RunState::kLabels;
  lc_status st = record(c);
  return st == LC_OK ? st : fail(c, st);
}

// Limits of the chunk-local grouping of lc_run_host: input chunks, and
// (bucket, chunk) runs, whose tile counts one block scans.
constexpr uint64_t kMaxGroupedChunks = 256;
constexpr uint64_t kMaxChunkSegments = 16384;

// Phase 0's steps that need only part of the input, run while the host edges
// are copied: the copies go chunk by chunk on a second stream, and each chunk,
// as soon as it has arrived, is grouped by vertex-block pair inside its own
// range of the grouped buffer (or, beyond the limits above, only counted for
// a grouping of all edges afterwards) and gets its share of the
// closed-neighbourhood minimum (atomic minima: any order of chunks gives the
// same minkey).  Everything after the minimum needs all edges; the relabel
// then walks the (bucket, chunk) runs in bucket order through a tile list.
static lc_status copy_input_overlapped(lc_ctx* c, const uint32_t* h_src, const uint32_t* h_dst) {
  const Launch& L = c->L;
  unsigned* err = &c->ctr->err;
  const uint64_t rk = phase_seed(c->seed, 0);
  if (!c->copy_stream &&
      cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return LC_ERR_CUDA;
  if (!c->copy_ev && cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming) != cudaSuccess)
    return LC_ERR_CUDA;
  init_keys(c->minkey, nullptr, c->n, rk, nullptr, L);
  const uint32_t nb = bucket_blocks(c, c->n);
  const uint64_t chunk = std::max<uint64_t>(c->host_chunk_edges, 1);
  const uint64_t chunks = (c->m + chunk - 1) / chunk;
  // group every chunk as it arrives (its scatter then runs under the copy)
  // when the chunks are few enough for their scratch and tile list; else
  // count the buckets per chunk and place all edges once they are in
  const uint64_t nbc = std::max<uint32_t>(2, std::min(nb, kBucketMaxBlocks));
  c->rs.pre0_chunks = 0;
  if (nb > 1 && chunks <= kMaxGroupedChunks && nbc * nbc * chunks <= kMaxChunkSegments) {
    const uint64_t sb = 4 * kChunkScratchWords * chunks;
    const uint64_t tb = chunk_tiles_bytes(c->m, nb, (uint32_t)chunks, kRelabelTileEdges) + 16;
    if (c->chunk_scratch_bytes < sb) {
      dev_free(c->mem, c->chunk_scratch);
      c->chunk_scratch_bytes = 0;
      if (dev_alloc(c->mem, &c->chunk_scratch, sb) != cudaSuccess) return LC_ERR_OOM;
      c->chunk_scratch_bytes = sb;
    }
    if (c->chunk_tile_bytes < tb) {
      dev_free(c->mem, c->chunk_tile_buf);
      c->chunk_tile_bytes = 0;
      if (dev_alloc(c->mem, &c->chunk_tile_buf, tb) != cudaSuccess) return LC_ERR_OOM;
      c->chunk_tile_bytes = tb;
    }
    c->rs.pre0_chunks = (uint32_t)chunks;
  } else if (nb > 1) {
    bucket_clear(c->n, nb, c->bucket_scratch, L);
  }
  // the copies may not overwrite the input before the work queued so far ends
  if (cudaEventRecord(c->copy_ev, c->stream) != cudaSuccess ||
      cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0) != cudaSuccess)
    return LC_ERR_CUDA;
  for (uint64_t off = 0; off < c->m; off += chunk) {
    const uint64_t len = std::min(chunk, c->m - off);
    if (cudaMemcpyAsync(c->own_src + off, h_src + off, len * 4, cudaMemcpyHostToDevice,
                        c->copy_stream) != cudaSuccess ||
        cudaMemcpyAsync(c->own_dst + off, h_dst + off, len * 4, cudaMemcpyHostToDevice,
                        c->copy_stream) != cudaSuccess ||
        cudaEventRecord(c->copy_ev, c->copy_stream) != cudaSuccess ||
        cudaStreamWaitEvent(c->stream, c->copy_ev, 0) != cudaSuccess)
      return LC_ERR_CUDA;
    if (c->rs.pre0_chunks > 0)
      bucket_edges(c->own_src + off, c->own_dst + off, len, c->n, nb, c->ebuf[1] + off,
                   c->chunk_scratch + (off / chunk) * kChunkScratchWords, err, L);
    else if (nb > 1)
      bucket_count(c->own_src + off, c->own_dst + off, len, c->n, nb, c->bucket_scratch, err, L);
    edge_min(c->own_src + off, c->own_dst + off, nullptr, len, c->n, rk, c->minkey, err,
             c->window_bytes, nullptr, L);
  }
  c->rs.pre0 = true;
  return LC_OK;
}

// Whether lc_run_host can overlap phase 0 with the input copy: a single graph
// whose phase 0 takes the closed-neighbourhood minimum.
static bool overlap_input(const lc_ctx* c) {
  return c->batch == nullptr && c->m > 0 && c->n > 0 &&
         (c->variant == LC_VARIANT_FOREST || c->variant == LC_VARIANT_TWO_HOP) &&
         !(c->finish_edges != 0 && c->m <= c->finish_edges);
}

static lc_status run_begin(lc_ctx* c, uint32_t* d_labels, const uint32_t* h_src = nullptr,
                           const uint32_t* h_dst = nullptr) {
  RunState& r = c->rs;
  r = RunState{};
  r.d_labels = d_labels;
  c->last_rounds = 0;
  c->last_mp.clear();
  c->last_emitted.clear();
  c->last_passes.clear();
  c->last_kept.clear();
  c->levels.clear();
  c->arena.reset();
  if (c->n == 0) {
    r.state = RunState::kDone;
    return LC_OK;
  }
  if (c->m == 0) {
    identity_labels(d_labels, c->n, c->L);
    if (c->batch) batch_localize(d_labels, c->n, c->batch->d_voff0, c->batch->k, c->L);
    c->h_ctr->err = 0;  // nothing below reads the device counters
    r.state = RunState::kLabels;
    lc_status st = record(c);
    return st == LC_OK ? st : fail(c, st);
  }
  if (cudaMemsetAsync(c->ctr, 0, sizeof(Counters), c->stream) != cudaSuccess)
    return fail(c, LC_ERR_CUDA);
  if (BatchState* b = c->batch) {
    b->voff.assign(1, b->d_voff0);
    b->mcnt.clear();
    batch_globalize(b->user_src, b->user_dst, b->d_eoff, b->d_voff0, b->k, c->m, c->own_src,
                    c->own_dst, &c->ctr->err, c->L);
    batch_graph_ids(b->d_voff0, b->k, c->n, b->d_gid, c->L);
  }
  cudaError_t aerr = cudaSuccess;
  r.ni = c->n;
  r.mi = c->m;
  r.packed = nullptr;
  r.mo_cur = c->arena.alloc(r.ni, &aerr);
  if (aerr != cudaSuccess) return fail(c, status_of(aerr));
  r.i = 0;
  if (h_src) {
    lc_status st = copy_input_overlapped(c, h_src, h_dst);
    if (st != LC_OK) return fail(c, st);
  }
  return enqueue_phase(c);
}

static lc_status run_wait(lc_ctx* c) {
  cudaError_t e = c->ev ? cudaEventSynchronize(c->ev) : cudaStreamSynchronize(c->stream);
  return status_of(e);
}

// Called once the work enqueued last has completed.
static lc_status report_internal(lc_ctx* c, const char* what) {
  const Counters& h = *c->h_ctr;
  std::fprintf(stderr,
               "liblc: %s: kernel %s index %llu limit %llu; phase %u of a graph with n = %u, "
               "m = %llu; phase n_i %u m_i %llu; counters m' %llu emitted %llu m_next %llu "
               "n_next %llu err %u tag %llu (expected %llu)\n",
               what, h.bad_kernel ? kernel_name((int)h.bad_kernel - 1) : "-",
               (unsigned long long)h.bad_index, (unsigned long long)h.bad_limit, c->rs.i, c->n,
               (unsigned long long)c->m, c->rs.ni, (unsigned long long)c->rs.mi, h.mprime,
               h.emitted, h.m_next, h.n_next, h.err, h.tag, (unsigned long long)c->tag);
  return fail(c, LC_ERR_INTERNAL);
}

static lc_status report_corrupt(lc_ctx* c) {
  return report_internal(c, "internal index check failed");
}

static lc_status run_complete(lc_ctx* c) {
  RunState& r = c->rs;
  c->prof.resolve();
  if (r.state == RunState::kLabels) {
    // the label kernels report index failures through the device error word
    if (c->h_ctr->tag != c->tag && c->m > 0) return report_internal(c, "stale counters");
    if (c->h_ctr->err & kErrCorrupt) return report_corrupt(c);
    c->last_rounds = (uint32_t)r.hn.size();  // phases (merge steps add levels, not phases)
    r.state = RunState::kDone;
    return LC_OK;
  }
  if (r.state != RunState::kPhase && r.state != RunState::kSortPhase &&
      r.state != RunState::kRelabel)
    return r.st;
  const Counters& h = *c->h_ctr;
  if (h.tag != c->tag) return report_internal(c, "stale counters");
  // a wait that ran out leaves later steps with unknown offsets, whose index
  // checks then fail too: the timeout is the cause to report
  if (h.err & kErrTimeout) return fail(c, LC_ERR_TIMEOUT);
  if (h.err & kErrCorrupt) return report_corrupt(c);
  if (h.err & kErrBadVertex) return fail(c, LC_ERR_INVALID);
  if (r.state == RunState::kRelabel) {
    // buckets of at most 1.5 kBucketTarget distinct keys on average (a 5%
    // margin on the estimate, whose standard error is 2.3%), which keeps the
    // bucket sets below three quarters full; never sized above the written keys
    if (h.emitted > r.mi || h.mprime > r.mi || (r.filtered && h.filtered > h.emitted))
      return report_internal(c, "inconsistent relabel counters");
    const uint64_t kept = r.filtered ? h.filtered : h.emitted;
    const double distinct = hll_estimate(c->h_hll) * (c->target_permille / 1000.0);
    if (r.seg) {
      // slices of at least 2.1 slots per estimated distinct key of a segment
      // (the estimate's standard error is 2.3%), a power of two each
      const double want = 2.1 * std::min(distinct, (double)kept) / kSegs;
      uint64_t slots = 64;
      while ((double)slots < want && slots < (1ull << 40)) slots <<= 1;
      if (enqueue_seg_dedup(c, slots)) return c->rs.state == RunState::kDone ? c->rs.st : LC_OK;
      // no room for the slices: the keys are contiguous again, partition them
    }
    const double est = distinct * 1.05 / 1.5 + 1.0;
    const uint64_t target = std::min<uint64_t>(std::max<uint64_t>(kept, 1),
                                               (uint64_t)std::min(est, (double)r.mi));
    PassPlan hplan{};
    const int hb = hash_plan(target, &hplan);
    return enqueue_dedup(c, hplan, hb, false);
  }
  if (r.state == RunState::kPhase && (h.err & kErrOverflow)) {
    // a bucket held more distinct keys than its shared-memory set: redo this
    // phase's deduplication by a full sort of the intact keys
    ++c->fallbacks;
    if (r.seg) {
      // the kept keys lie in segment regions: make them contiguous first
      seg_compact(r.part, c->bucket_scratch, r.next, c->L);
      std::swap(r.part, r.next);
      r.seg = false;
    }
    unmix_keys(r.part, kept_count(c), r.mi, c->L);
    if (cudaMemsetAsync(&c->ctr->m_next, 0, 2 * sizeof(unsigned long long), c->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(&c->ctr->err, 0, sizeof(unsigned), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->flags, 0, 4 * flag_words(r.ni), c->stream) != cudaSuccess)
      return fail(c, LC_ERR_CUDA);
    r.state = RunState::kSortPhase;
    lc_status st = enqueue_sort_dedup(c);
    if (st != LC_OK) return st;
    stamp_counters(c->ctr, ++c->tag, c->L);
    if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
      return fail(c, LC_ERR_CUDA);
    st = record(c);
    return st == LC_OK ? st : fail(c, st);
  }
  if ((h.n_next > 0) != (h.m_next > 0) || h.n_next > r.ni || h.m_next > h.emitted)
    return report_internal(c, "inconsistent phase counters");
  const bool was_merge = r.merge_step;
  if (!was_merge) {
    r.hn.push_back(r.ni);
    r.hm.push_back(r.mi);
    c->last_mp.push_back(h.mprime);
    c->last_emitted.push_back(h.emitted);
    c->last_passes.push_back(r.passes);
    c->last_kept.push_back(r.filtered ? h.filtered : h.emitted);
  }
  const bool finished_by_uf = !was_merge && c->finish_edges != 0 && r.mi <= c->finish_edges;
  c->levels.push_back(r.lv);
  r.ni = (uint32_t)h.n_next;
  r.mi = h.m_next;
  r.packed = r.next;
  r.mo_cur = r.mo_next;
  r.merge_step = false;
  if (r.mi == 0) return enqueue_labels(c);
  if (!was_merge && !finished_by_uf && r.i < c->merge_alpha.size() && c->merge_alpha[r.i] > 0) {
    // the phase's MergeToLarge step: one more contraction level, same phase
    r.merge_step = true;
    return enqueue_phase(c);
  }
  if (++r.i >= (c->max_rounds ? c->max_rounds : round_cap(c->n)))
    return fail(c, LC_ERR_NO_CONVERGENCE);
  return enqueue_phase(c);
}

static lc_status run_loop(lc_ctx* c, uint32_t* d_labels, uint32_t* rounds, uint64_t* n_i,
                          uint64_t* m_i, uint32_t cap, const uint32_t* h_src = nullptr,
                          const uint32_t* h_dst = nullptr) {
  if (rounds) *rounds = 0;
  lc_status st = run_begin(c, d_labels, h_src, h_dst);
  while (st == LC_OK && c->rs.state != RunState::kDone) {
    st = run_wait(c);
    if (st == LC_OK) st = run_complete(c);
  }
  if (st != LC_OK) return st;
  const uint32_t R = c->last_rounds;
  if (rounds) *rounds = R;
  if (n_i || m_i) {
    for (uint32_t i = 0; i < std::min(R, cap); ++i) {
      if (n_i) n_i[i] = c->rs.hn[i];
      if (m_i) m_i[i] = c->rs.hm[i];
    }
    if (R > cap) return LC_ERR_INVALID;
  }
  return LC_OK;
}

extern "C" lc_status lc_run(lc_ctx* c, uint32_t* d_labels, uint32_t* rounds, uint64_t* n_i,
                            uint64_t* m_i, uint32_t cap) {
  if (!c || (!d_labels && c->n > 0)) return LC_ERR_INVALID;
  DeviceGuard g(c->device);
  return run_loop(c, d_labels, rounds, n_i, m_i, cap);
}

extern "C" lc_status lc_run_host(lc_ctx* c, const uint32_t* h_src, const uint32_t* h_dst,
                                 uint32_t* h_labels, uint32_t* rounds, uint64_t* n_i,
                                 uint64_t* m_i, uint32_t cap) {
  if (!c || !c->own_src) return LC_ERR_INVALID;
  if (c->m > 0 && (!h_src || !h_dst)) return LC_ERR_INVALID;
  if (c->n > 0 && !h_labels) return LC_ERR_INVALID;
  DeviceGuard g(c->device);
  lc_status st;
  if (overlap_input(c)) {
    st = run_loop(c, c->own_labels, rounds, n_i, m_i, cap, h_src, h_dst);
  } else {
    if (c->m > 0) {
      LC_TRY(cudaMemcpyAsync(c->own_src, h_src, c->m * 4, cudaMemcpyHostToDevice, c->stream));
      LC_TRY(cudaMemcpyAsync(c->own_dst, h_dst, c->m * 4, cudaMemcpyHostToDevice, c->stream));
    }
    st = run_loop(c, c->own_labels, rounds, n_i, m_i, cap);
  }
  if (st != LC_OK && st != LC_ERR_INVALID) return st;
  if (c->n > 0) {
    LC_TRY(cudaMemcpyAsync(h_labels, c->own_labels, (uint64_t)c->n * 4, cudaMemcpyDeviceToHost,
                           c->stream));
    LC_TRY(cudaStreamSynchronize(c->stream));
  }
  return st;
}

extern "C" lc_status lc_batch_create(uint32_t k, const uint32_t* h_n, const uint64_t* h_eoff,
                                     const uint32_t* d_src, const uint32_t* d_dst,
                                     const uint64_t* h_seeds, void* stream, lc_ctx** out) {
  if (!out) return LC_ERR_INVALID;
  *out = nullptr;
  if (k == 0 || !h_n || !h_eoff || !h_seeds) return LC_ERR_INVALID;
  if (h_eoff[0] != 0) return LC_ERR_INVALID;
  std::vector<uint32_t> voff(k + 1, 0);
  uint64_t tot = 0;
  for (uint32_t g = 0; g < k; ++g) {
    if (h_eoff[g + 1] < h_eoff[g]) return LC_ERR_INVALID;
    if (h_eoff[g + 1] > h_eoff[g] && h_n[g] == 0) return LC_ERR_INVALID;
    tot += h_n[g];
    if (tot > 0xFFFFFFFFull) return LC_ERR_INVALID;
    voff[g + 1] = (uint32_t)tot;
  }
  const uint64_t m = h_eoff[k];
  if (m > 0xFFFFFFFFull || (m > 0 && (!d_src || !d_dst))) return LC_ERR_INVALID;
  // the context owns the global-id copy of the edges (filled at every run)
  lc_ctx* c = nullptr;
  lc_status st = lc_create((uint32_t)tot, nullptr, nullptr, m, 0, stream, &c);
  if (st != LC_OK) return st;
  BatchState* b = new (std::nothrow) BatchState();
  if (!b) {
    lc_destroy(c);
    return LC_ERR_OOM;
  }
  c->batch = b;
  b->k = k;
  b->user_src = d_src;
  b->user_dst = d_dst;
  b->h_eoff.assign(h_eoff, h_eoff + k + 1);
  b->h_voff0 = voff;
  cudaError_t e = dev_alloc(c->mem, &b->d_seeds, 8ull * k);
  if (e == cudaSuccess) e = dev_alloc(c->mem, &b->d_voff0, 4ull * (k + 1));
  if (e == cudaSuccess) e = dev_alloc(c->mem, &b->d_eoff, 8ull * (k + 1));
  if (e == cudaSuccess) e = dev_alloc(c->mem, &b->d_rk, 8ull * k);
  if (e == cudaSuccess) e = dev_alloc(c->mem, &b->d_gid, 4ull * std::max<uint64_t>(tot, 1));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_seeds, h_seeds, 8ull * k, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_voff0, voff.data(), 4ull * (k + 1), cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_eoff, h_eoff, 8ull * (k + 1), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  // level arrays of a batch: offsets and edge counts per graph per level
  if (e == cudaSuccess) e = c->arena.init(64ull * (2 * k + 2));
  if (e != cudaSuccess) {
    lc_destroy(c);
    return status_of(e);
  }
  *out = c;
  return LC_OK;
}

extern "C" lc_status lc_batch_run(lc_ctx* c, uint32_t* d_labels, uint32_t* rounds,
                                  uint64_t* n_i, uint64_t* m_i, uint32_t cap) {
  if (!c || !c->batch || (!d_labels && c->n > 0)) return LC_ERR_INVALID;
  DeviceGuard g(c->device);
  BatchState* b = c->batch;
  lc_status st = run_loop(c, d_labels, nullptr, nullptr, nullptr, 0);
  if (st != LC_OK) return st;
  const uint32_t k = b->k, R = c->last_rounds;
  // per-level per-graph sizes: level 0 from the input, later levels from the
  // device arrays written during the run
  std::vector<uint32_t> voff(k + 1), mcnt(k);
  std::vector<uint32_t> Rg(k, 0);
  bool over = false;
  for (uint32_t i = 0; i < R; ++i) {
    if (i == 0) {
      voff = b->h_voff0;
      for (uint32_t gi = 0; gi < k; ++gi) mcnt[gi] = (uint32_t)(b->h_eoff[gi + 1] - b->h_eoff[gi]);
    } else {
      LC_TRY(cudaMemcpyAsync(voff.data(), b->voff[i], 4ull * (k + 1), cudaMemcpyDeviceToHost,
                             c->stream));
      LC_TRY(cudaMemcpyAsync(mcnt.data(), b->mcnt[i - 1], 4ull * k, cudaMemcpyDeviceToHost,
                             c->stream));
      LC_TRY(cudaStreamSynchronize(c->stream));
    }
    for (uint32_t gi = 0; gi < k; ++gi) {
      if (mcnt[gi] == 0) continue;  // graph finished before this phase
      if (Rg[gi] != i) continue;     // (cannot happen: a finished graph stays finished)
      if (i < cap) {
        if (n_i) n_i[(uint64_t)gi * cap + i] = voff[gi + 1] - voff[gi];
        if (m_i) m_i[(uint64_t)gi * cap + i] = mcnt[gi];
      } else {
        over = true;
      }
      Rg[gi] = i + 1;
    }
  }
  if (rounds)
    for (uint32_t gi = 0; gi < k; ++gi) rounds[gi] = Rg[gi];
  return over ? LC_ERR_INVALID : LC_OK;
}

extern "C" lc_status lc_last_stats(const lc_ctx* c, uint32_t* rounds, uint64_t* mp_i,
                                   uint64_t* emitted_i, uint32_t cap) {
  if (!c) return LC_ERR_INVALID;
  if (rounds) *rounds = c->last_rounds;
  for (uint32_t i = 0; i < std::min<uint32_t>(cap, (uint32_t)c->last_mp.size()); ++i) {
    if (mp_i) mp_i[i] = c->last_mp[i];
    if (emitted_i) emitted_i[i] = c->last_emitted[i];
  }
  return LC_OK;
}

extern "C" lc_status lc_last_dedup(const lc_ctx* c, uint32_t* rounds, uint64_t* kept_i,
                                   uint32_t* passes_i, uint32_t cap) {
  if (!c) return LC_ERR_INVALID;
  if (rounds) *rounds = c->last_rounds;
  for (uint32_t i = 0; i < std::min<uint32_t>(cap, (uint32_t)c->last_passes.size()); ++i) {
    if (kept_i) kept_i[i] = c->last_kept[i];
    if (passes_i) passes_i[i] = c->last_passes[i];
  }
  return c->last_passes.size() > cap ? LC_ERR_INVALID : LC_OK;
}

extern "C" lc_status lc_dedup_fallbacks(const lc_ctx* c, uint64_t* count) {
  if (!c || !count) return LC_ERR_INVALID;
  *count = c->fallbacks;
  return LC_OK;
}

extern "C" lc_status lc_set_dedup(lc_ctx* c, lc_dedup mode) {
  if (!c) return LC_ERR_INVALID;
  if (mode != LC_DEDUP_HASH && mode != LC_DEDUP_SORT) return LC_ERR_INVALID;
  c->dedup_sort = mode == LC_DEDUP_SORT;
  return LC_OK;
}

extern "C" lc_status lc_set_param(lc_ctx* c, const char* name, uint64_t value) {
  if (!c || !name) return LC_ERR_INVALID;
  if (std::strcmp(name, "window_bytes") == 0) {
    if (value < (1u << 20)) return LC_ERR_INVALID;
    c->window_bytes = value;
    return LC_OK;
  }
  if (std::strcmp(name, "max_rounds") == 0) {
    if (value > (1u << 20)) return LC_ERR_INVALID;
    c->max_rounds = (uint32_t)value;
    return LC_OK;
  }
  if (std::strcmp(name, "spin_limit") == 0) {
    if (value == 0 || value > (1u << 30)) return LC_ERR_INVALID;
    c->sort.spin_limit = (uint32_t)value;
    return LC_OK;
  }
  if (std::strcmp(name, "inject_lookback_stall") == 0) {
    if (value > 1) return LC_ERR_INVALID;
    c->sort.stall_once = (int)value;
    return LC_OK;
  }
  if (std::strcmp(name, "cache_in_relabel") == 0) {
    if (value > 1) return LC_ERR_INVALID;
    c->cache_in_relabel = value != 0;
    return LC_OK;
  }
  if (std::strcmp(name, "jump_bits_min_vertices") == 0) {
    if (value == 0 || value > 0xFFFFFFFFull) return LC_ERR_INVALID;
    c->jump_bits_min_vertices = (uint32_t)value;
    return LC_OK;
  }
  if (std::strcmp(name, "seg_dedup") == 0) {
    if (value > 1) return LC_ERR_INVALID;
    c->seg_dedup = value != 0;
    return LC_OK;
  }
  if (std::strcmp(name, "table_slots") == 0) {
    if (value != 0 && (value < (uint64_t)kSegs * 64 || (value & (value - 1)) != 0))
      return LC_ERR_INVALID;
    c->table_cap = value;
    return LC_OK;
  }
  if (std::strcmp(name, "target_permille") == 0) {
    if (value == 0 || value > 1000000) return LC_ERR_INVALID;
    c->target_permille = (uint32_t)value;
    return LC_OK;
  }
  if (std::strcmp(name, "late_min_edges") == 0) {
    if (value < 1024) return LC_ERR_INVALID;
    if (c->rs.state != RunState::kDone) return LC_ERR_INVALID;
    if (value < c->m_cap && (c->d_hll == nullptr || c->dtable == nullptr)) {
      DeviceGuard g(c->device);
      LC_TRY(cudaStreamSynchronize(c->stream));
      LC_TRY(alloc_late(c));
    }
    c->late_min_edges = value;
    return LC_OK;
  }
  if (std::strcmp(name, "host_chunk_edges") == 0) {
    if (value == 0 || value > 0xFFFFFFFFull) return LC_ERR_INVALID;
    c->host_chunk_edges = value;
    return LC_OK;
  }
  if (std::strcmp(name, "bucket_blocks") == 0) {
    if (value > kBucketMaxBlocks) return LC_ERR_INVALID;
    c->bucket_blocks = (uint32_t)value;
    return LC_OK;
  }
  if (std::strcmp(name, "bucket_window_bytes") == 0) {
    if (value < (1u << 20)) return LC_ERR_INVALID;
    c->bucket_window_bytes = value;
    return LC_OK;
  }
  if (std::strcmp(name, "bucket_min_vertices") == 0) {
    if (value > 0xFFFFFFFFull) return LC_ERR_INVALID;
    c->bucket_min_vertices = (uint32_t)value;
    return LC_OK;
  }
  if (std::strcmp(name, "relabel_window_bytes") == 0) {
    c->relabel_window_bytes = value;
    return LC_OK;
  }
  if (std::strcmp(name, "relabel_cache_admit") == 0) {
    if (value > 16) return LC_ERR_INVALID;
    c->gcache_admit = (int)value;
    return LC_OK;
  }
  if (std::strcmp(name, "relabel_cache_slots") == 0) {
    if (value != 0 && (value < 1024 || value > (1ull << 26) || (value & (value - 1)) != 0))
      return LC_ERR_INVALID;
    if (c->rs.state != RunState::kDone) return LC_ERR_INVALID;
    DeviceGuard g(c->device);
    LC_TRY(cudaStreamSynchronize(c->stream));
    dev_free(c->mem, c->gcache);
    c->gcache = nullptr;
    c->gcache_slots = 0;
    if (value != 0) {
      LC_TRY(dev_alloc(c->mem, &c->gcache, 8ull * value));
      c->gcache_slots = (uint32_t)value;
    }
    return LC_OK;
  }
  return LC_ERR_INVALID;
}

extern "C" lc_status lc_profile(lc_ctx* c, int on) {
  if (!c) return LC_ERR_INVALID;
  DeviceGuard g(c->device);
  LC_TRY(cudaStreamSynchronize(c->stream));
  c->prof.resolve();
  c->prof.reset();
  c->prof.on = on != 0;
  return LC_OK;
}

extern "C" lc_status lc_kernel_stats(const lc_ctx* c, uint32_t k, const char** name,
                                     uint64_t* launches, double* ms) {
  if (!c || k >= (uint32_t)kNumKernels) return LC_ERR_INVALID;
  if (name) *name = kernel_name((int)k);
  if (launches) *launches = c->prof.launches[k];
  if (ms) *ms = c->prof.ms[k];
  return LC_OK;
}

extern "C" lc_status lc_destroy(lc_ctx* c) {
  if (!c) return LC_OK;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  return LC_OK;
}

extern "C" const char* lc_status_str(lc_status s) {
  switch (s) {
    case LC_OK: return "ok";
    case LC_ERR_INVALID: return "invalid argument or input";
    case LC_ERR_OOM: return "device allocation failed";
    case LC_ERR_CUDA: return "CUDA runtime error";
    case LC_ERR_NO_CONVERGENCE: return "phase count exceeded the round cap";
    case LC_ERR_TIMEOUT: return "a bounded device wait gave up";
    case LC_ERR_INTERNAL: return "internal consistency check failed";
    case LC_ERR_CANCELLED: return "the job was cancelled";
  }
  return "unknown status";
}

extern "C" lc_status lc_rank_probe(uint64_t seed, uint32_t i, uint32_t v0, uint32_t count,
                                   uint32_t* d_out, void* stream) {
  if (count > 0 && !d_out) return LC_ERR_INVALID;
  Launch L{(cudaStream_t)stream, 1};
  int dev = 0;
  LC_TRY(cudaGetDevice(&dev));
  LC_TRY(cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev));
  rank_probe(phase_seed(seed, i), v0, count, d_out, L);
  LC_TRY(cudaGetLastError());
  return LC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot call cudaMalloc: code running under another
// framework's caching allocator that already holds the device memory, plug-ins
// and callbacks that must not touch the allocator, and latency-critical loops
// that avoid cudaMalloc because it can synchronise the device.  lc_run_static
// runs the same phase loop as lc_run for small graphs with every scratch
// buffer carved out of one file-scope device array.  Every GPU that loads
// the library holds that array until the process exits.

static __device__ __align__(256) unsigned char g_static_scratch[LC_STATIC_SCRATCH_BYTES];

namespace {

// Layout of the static array (byte offsets, 256-byte aligned pieces).
constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }
constexpr uint64_t kSN = LC_STATIC_MAX_N, kSM = LC_STATIC_MAX_M;
constexpr uint64_t kOffMinkey = 0;
constexpr uint64_t kOffFlags = align256(kOffMinkey + 8 * kSN);
constexpr uint64_t kOffEbuf0 = align256(kOffFlags + 4 * (flag_words(kSN) + 4));
constexpr uint64_t kOffEbuf1 = align256(kOffEbuf0 + 8 * kSM);
constexpr uint64_t kOffCtr = align256(kOffEbuf1 + 8 * kSM);
constexpr uint64_t kStatusWords = (kSM + kSortTile - 1) / kSortTile * kRadixMax + 1024;
constexpr uint64_t kOffStatus = align256(kOffCtr + sizeof(Counters));
constexpr uint64_t kOffHist = align256(kOffStatus + 8 * kStatusWords);
constexpr uint64_t kOffTickets = align256(kOffHist + 4ull * kMaxPasses * kRadixMax);
constexpr uint64_t kBoundsWords = (1ull << 8) + 1;  // hash_bits_for(LC_STATIC_MAX_M) == 8
constexpr uint64_t kOffBounds = align256(kOffTickets + 4 * 16);
constexpr uint64_t kOffArena = align256(kOffBounds + 4 * kBoundsWords);
constexpr uint64_t kArenaWords = (LC_STATIC_SCRATCH_BYTES - kOffArena) / 4;
static_assert(kOffArena < LC_STATIC_SCRATCH_BYTES, "static scratch too small");
static_assert(kArenaWords >= 16 * kSN, "static level arena below 16 words per vertex");

constexpr int kMaxStaticDevices = 64;
unsigned char* g_static_base[kMaxStaticDevices];  // device address, per device
std::mutex g_static_mu;

// Device address of the static array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked
// up once per device with that device current.
lc_status static_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxStaticDevices) return LC_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_base[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return status_of(e);
    g_static_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_static_base[dev];
  return LC_OK;
}

}  // namespace

extern "C" lc_status lc_run_static(uint32_t n, const uint32_t* d_src, const uint32_t* d_dst,
                                   uint64_t m, uint64_t seed, void* stream, uint32_t* d_labels,
                                   uint32_t* rounds, uint64_t* n_i, uint64_t* m_i, uint32_t cap) {
  if (n > LC_STATIC_MAX_N || m > LC_STATIC_MAX_M) return LC_ERR_INVALID;  // too large
  if ((1ull << hash_bits_for(m)) + 1 > kBoundsWords) return LC_ERR_INVALID;
  if (n == 0 && m > 0) return LC_ERR_INVALID;
  if (m > 0 && (d_src == nullptr || d_dst == nullptr)) return LC_ERR_INVALID;
  if (n > 0 && d_labels == nullptr) return LC_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LC_ERR_CUDA;
  unsigned char* base = nullptr;
  lc_status st = static_scratch(dev, &base);
  if (st != LC_OK) return st;
  lc_ctx c;  // host-side bookkeeping only; every device buffer points into base
  c.n = n;
  c.m = m;
  c.seed = seed;
  c.stream = (cudaStream_t)stream;
  c.device = dev;
  if (cudaDeviceGetAttribute(&c.L.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LC_ERR_CUDA;
  c.L.stream = c.stream;
  c.L.prof = &c.prof;
  c.src = d_src;
  c.dst = d_dst;
  c.minkey = reinterpret_cast<unsigned long long*>(base + kOffMinkey);
  c.flags = reinterpret_cast<uint32_t*>(base + kOffFlags);
  c.ebuf[0] = reinterpret_cast<uint64_t*>(base + kOffEbuf0);
  c.ebuf[1] = reinterpret_cast<uint64_t*>(base + kOffEbuf1);
  c.ctr = reinterpret_cast<Counters*>(base + kOffCtr);
  Counters host_ctr;
  c.h_ctr = &host_ctr;
  c.sort.status = reinterpret_cast<uint64_t*>(base + kOffStatus);
  c.sort.status_words = kStatusWords;
  c.sort.hist = reinterpret_cast<uint32_t*>(base + kOffHist);
  c.sort.tickets = reinterpret_cast<unsigned*>(base + kOffTickets);
  c.sort.epoch = 0;  // the array keeps the last call's words: clear them on first use
  c.bounds = reinterpret_cast<uint32_t*>(base + kOffBounds);
  c.arena.chunks.push_back({reinterpret_cast<uint32_t*>(base + kOffArena), kArenaWords});
  c.arena.fixed = true;
  // the run clears the counters, status words, histograms, tickets and
  // flags it reads before reading them
  st = run_loop(&c, d_labels, rounds, n_i, m_i, cap);
  c.arena.chunks.clear();  // nothing to free: all of it is the static array
  return st;
}

// ---------------------------------------------------------------------------
// Serving: a request loop with continuous batching (native worker thread).
//
// Jobs (one graph each, host edge arrays) are admitted in arrival order while
// the device-memory budget and the number of slots allow.  Each admitted job
// gets a context (reused from a pool of idle contexts when one is large
// enough, so steady-state admission allocates nothing) and its slot's CUDA
// stream; its contracted graph stays on the device between phases.  The
// worker polls every running job's last event and enqueues that job's next
// phase as soon as the previous one completes, so phases of different jobs
// interleave and overlap on the device, and jobs that arrive while others run
// are admitted as soon as a slot and memory free up.

namespace {

// Device bytes of a context allocated for (n, m) with its own input buffers
// (mirrors alloc_ctx and lc_create).
uint64_t ctx_bytes(uint64_t n, uint64_t m) {
  const uint64_t status = std::max(sort_status_words(m), sort_status_words(n)) * 8;
  const uint64_t bounds = 4 * ((1ull << hash_bits_for(m)) + 1);
  const uint64_t arena = 4 * std::max<uint64_t>(4 * (2 * n + 256), 1024);
  const uint64_t gcache =
      m >= kGCacheMinEdges ? 8ull * kGCacheSlots + 4ull * kHllRegs + 8 * table_slots_for(m) : 0;
  return gcache + 8 * std::max<uint64_t>(n, 1) + 4 * (flag_words(n) + 4) + 16 * std::max<uint64_t>(m, 2) + status +
         bounds + arena + 8 * std::max<uint64_t>(m, 1) + 4 * std::max<uint64_t>(n, 1) +
         sizeof(Counters) + 4096 + 16 * 4 + 4ull * kMaxPasses * kRadixMax + (1u << 16) +
         4 * kBucketScratchWords;
}

struct Job {
  uint64_t id = 0;
  uint32_t n = 0;
  uint64_t m = 0, seed = 0;
  const uint32_t *h_src = nullptr, *h_dst = nullptr;
  uint32_t* h_labels = nullptr;
  enum { kQueued, kRunning, kCopying, kDone } state = kQueued;
  lc_status status = LC_OK;
  bool cancel = false;  // stop at the next phase boundary
  uint32_t rounds = 0;
  std::vector<uint64_t> hn, hm;  // per-phase sizes of a finished run
  lc_ctx* ctx = nullptr;
  int slot = -1;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

}  // namespace

struct lc_server {
  std::vector<lc_ctx*> in_use_ctx;  // contexts held by running jobs (consistency check)
  int device = 0;
  cudaMemPool_t mempool = nullptr;  // device memory of the server's contexts
  std::vector<unsigned char*> pinned_chunks, pinned_free;  // host counter blocks
  uint64_t budget = 0, in_use = 0;
  std::vector<cudaStream_t> streams;
  std::vector<int> free_slots;
  std::vector<lc_ctx*> pool;  // idle contexts
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::unordered_map<uint64_t, Job*> jobs;
  uint64_t next_id = 1, completed = 0, peak_active = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
};

// Re-bind an idle context (allocated with its own inputs for at least n
// vertices and m edges) to a new graph of that size.
static void ctx_rebind(lc_ctx* c, uint32_t n, uint64_t m, uint64_t seed, cudaStream_t stream) {
  c->n = n;
  c->m = m;
  c->seed = seed;
  c->stream = stream;
  c->mem.stream = stream;
  c->L.stream = stream;
  c->src = c->own_src;
  c->dst = c->own_dst;
}

// A pinned block for a new context's host counters (the server allocates
// them 64 at a time and never returns them before it is destroyed).
static unsigned char* take_pinned(lc_server* s) {
  if (s->pinned_free.empty()) {
    constexpr int kPer = 64;
    unsigned char* chunk = nullptr;
    if (host_alloc(&chunk, kPinnedBlock * kPer) != cudaSuccess) return nullptr;
    s->pinned_chunks.push_back(chunk);
    for (int q = kPer - 1; q >= 0; --q) s->pinned_free.push_back(chunk + kPinnedBlock * q);
  }
  unsigned char* b = s->pinned_free.back();
  s->pinned_free.pop_back();
  return b;
}

// Release an idle (or failed) context of the server: all its work has
// completed, so its memory goes back to the pool stream-ordered, without
// waiting on the device.
static void server_release(lc_server* s, lc_ctx* c) {
  if (c->pinned) s->pinned_free.push_back(c->pinned);
  free_ctx(c);
}

static void finish_job(lc_server* s, Job* j, lc_status st) {
  j->status = st;
  j->state = Job::kDone;
  j->t_done = std::chrono::steady_clock::now();
  if (j->ctx) {
    auto it = std::find(s->in_use_ctx.begin(), s->in_use_ctx.end(), j->ctx);
    if (it != s->in_use_ctx.end()) s->in_use_ctx.erase(it);
    if (std::find(s->pool.begin(), s->pool.end(), j->ctx) != s->pool.end())
      std::fprintf(stderr, "liblc: server: context returned to the pool twice\n");
    if (st == LC_OK || st == LC_ERR_INVALID || st == LC_ERR_NO_CONVERGENCE ||
        st == LC_ERR_CANCELLED) {
      j->ctx->rs.state = RunState::kDone;
      s->pool.push_back(j->ctx);  // the context is intact: keep it for reuse
    } else {
      s->in_use -= ctx_bytes(j->ctx->n_cap, j->ctx->m_cap);
      server_release(s, j->ctx);
    }
    j->ctx = nullptr;
  }
  if (j->slot >= 0) s->free_slots.push_back(j->slot);
  j->slot = -1;
  ++s->completed;
}

// Admit queued jobs while a slot is free and their memory fits.  Called with
// the lock held; returns whether anything was admitted.
static bool admit(lc_server* s) {
  bool any = false;
  while (!s->queue.empty() && !s->free_slots.empty()) {
    Job* j = s->queue.front();
    // best-fitting idle context
    int best = -1;
    for (size_t q = 0; q < s->pool.size(); ++q) {
      lc_ctx* c = s->pool[q];
      if (c->n_cap >= j->n && c->m_cap >= j->m &&
          (best < 0 || ctx_bytes(c->n_cap, c->m_cap) <
                           ctx_bytes(s->pool[best]->n_cap, s->pool[best]->m_cap)))
        best = (int)q;
    }
    lc_ctx* c = nullptr;
    if (best >= 0) {
      c = s->pool[best];
      s->pool.erase(s->pool.begin() + best);
    } else {
      const uint64_t need = ctx_bytes(j->n, j->m);
      // release idle contexts (largest first) until the new one fits
      while (s->in_use + need > s->budget && !s->pool.empty()) {
        auto it = std::max_element(s->pool.begin(), s->pool.end(), [](lc_ctx* a, lc_ctx* b) {
          return ctx_bytes(a->n_cap, a->m_cap) < ctx_bytes(b->n_cap, b->m_cap);
        });
        s->in_use -= ctx_bytes((*it)->n_cap, (*it)->m_cap);
        server_release(s, *it);
        s->pool.erase(it);
      }
      if (s->in_use + need > s->budget) break;  // wait for running jobs to free memory
      // created on the slot's stream, from the server's pool: no device-wide
      // synchronisation on the worker's path
      unsigned char* pin = take_pinned(s);
      lc_status st = pin == nullptr ? LC_ERR_OOM
                                    : create_ctx(j->n, nullptr, nullptr, j->m, j->seed,
                                                 s->streams[s->free_slots.back()], s->mempool, pin,
                                                 &c);
      if (st != LC_OK && pin != nullptr) s->pinned_free.push_back(pin);
      if (st != LC_OK) {
        s->queue.pop_front();
        finish_job(s, j, st);
        any = true;
        continue;
      }
      s->in_use += need;
    }
    s->queue.pop_front();
    j->slot = s->free_slots.back();
    s->free_slots.pop_back();
    if (std::find(s->in_use_ctx.begin(), s->in_use_ctx.end(), c) != s->in_use_ctx.end())
      std::fprintf(stderr, "liblc: server: context given to two running jobs\n");
    s->in_use_ctx.push_back(c);
    j->ctx = c;
    ctx_rebind(c, j->n, j->m, j->seed, s->streams[j->slot]);
    lc_status st = LC_OK;
    if (j->m > 0) {
      if (cudaMemcpyAsync(c->own_src, j->h_src, j->m * 4, cudaMemcpyHostToDevice, c->stream) !=
              cudaSuccess ||
          cudaMemcpyAsync(c->own_dst, j->h_dst, j->m * 4, cudaMemcpyHostToDevice, c->stream) !=
              cudaSuccess)
        st = LC_ERR_CUDA;
    }
    if (st == LC_OK) st = run_begin(c, c->own_labels);
    if (st != LC_OK) {
      finish_job(s, j, st);
    } else {
      j->state = Job::kRunning;
      s->active.push_back(j);
      s->peak_active = std::max<uint64_t>(s->peak_active, s->active.size());
    }
    any = true;
  }
  return any;
}

// Advance every running job whose last enqueued work has completed.  A CUDA
// error while polling fails the job (LC_ERR_CUDA) instead of leaving it
// running.
static bool progress(lc_server* s) {
  bool any = false;
  for (size_t q = 0; q < s->active.size();) {
    Job* j = s->active[q];
    lc_ctx* c = j->ctx;
    bool finished = false;
    if (j->state == Job::kRunning) {
      cudaError_t e = c->rs.state == RunState::kDone ? cudaSuccess : cudaEventQuery(c->ev);
      if (e == cudaSuccess && j->cancel) {
        // the work enqueued last has completed: stop at this phase boundary
        finish_job(s, j, LC_ERR_CANCELLED);
        finished = true;
        any = true;
      } else if (e == cudaSuccess) {
        lc_status st = c->rs.state == RunState::kDone ? c->rs.st : run_complete(c);
        if (st != LC_OK) {
          finish_job(s, j, st);
          finished = true;
        } else if (c->rs.state == RunState::kDone) {
          j->rounds = c->last_rounds;
          j->hn = c->rs.hn;
          j->hm = c->rs.hm;
          if (j->n > 0 &&
              (cudaMemcpyAsync(j->h_labels, c->own_labels, (uint64_t)j->n * 4,
                               cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
               cudaEventRecord(c->ev, c->stream) != cudaSuccess)) {
            finish_job(s, j, LC_ERR_CUDA);
            finished = true;
          } else {
            j->state = Job::kCopying;
          }
        }
        any = true;
      } else if (e != cudaErrorNotReady) {
        finish_job(s, j, LC_ERR_CUDA);
        finished = true;
        any = true;
      }
    } else if (j->state == Job::kCopying) {
      cudaError_t e = j->n == 0 ? cudaSuccess : cudaEventQuery(c->ev);
      if (e != cudaErrorNotReady) {
        finish_job(s, j, e == cudaSuccess ? LC_OK : LC_ERR_CUDA);
        finished = true;
        any = true;
      }
    }
    if (finished) {
      s->active.erase(s->active.begin() + q);
    } else {
      ++q;
    }
  }
  return any;
}

static void serve(lc_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    if (s->stop && s->queue.empty() && s->active.empty()) break;
    bool any = admit(s);
    any = progress(s) || any;
    if (any) s->cv_done.notify_all();
    if (s->active.empty() && (s->queue.empty() || s->free_slots.empty())) {
      s->cv_work.wait(lock);
    } else if (!any) {
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lock.lock();
    }
  }
}

extern "C" lc_status lc_server_create(uint64_t budget_bytes, uint32_t slots, lc_server** out) {
  if (!out || slots == 0 || slots > 1024) return LC_ERR_INVALID;
  *out = nullptr;
  lc_server* s = new (std::nothrow) lc_server();
  if (!s) return LC_ERR_OOM;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return LC_ERR_CUDA;
  }
  if (budget_bytes == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete s;
      return LC_ERR_CUDA;
    }
    budget_bytes = (uint64_t)(free_b * 0.8);
  }
  s->budget = budget_bytes;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if (cudaMemPoolCreate(&s->mempool, &props) != cudaSuccess) {
    delete s;
    return LC_ERR_CUDA;
  }
  // keep released memory in the pool for later contexts (up to the budget)
  uint64_t keep = budget_bytes;
  cudaMemPoolSetAttribute(s->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
  for (uint32_t q = 0; q < slots; ++q) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      cudaMemPoolDestroy(s->mempool);
      delete s;
      return LC_ERR_CUDA;
    }
    s->streams.push_back(st);
    s->free_slots.push_back((int)(slots - 1 - q));
  }
  s->worker = std::thread(serve, s);
  *out = s;
  return LC_OK;
}

extern "C" lc_status lc_server_submit(lc_server* s, uint32_t n, const uint32_t* h_src,
                                      const uint32_t* h_dst, uint64_t m, uint64_t seed,
                                      uint32_t* h_labels, uint64_t* job) {
  if (!s || !job) return LC_ERR_INVALID;
  if (m > 0xFFFFFFFFull || (n == 0 && m > 0)) return LC_ERR_INVALID;
  if ((m > 0 && (!h_src || !h_dst)) || (n > 0 && !h_labels)) return LC_ERR_INVALID;
  if (ctx_bytes(n, m) > s->budget) return LC_ERR_OOM;  // could never be admitted
  Job* j = new (std::nothrow) Job();
  if (!j) return LC_ERR_OOM;
  j->n = n;
  j->m = m;
  j->seed = seed;
  j->h_src = h_src;
  j->h_dst = h_dst;
  j->h_labels = h_labels;
  j->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) {
      delete j;
      return LC_ERR_INVALID;
    }
    j->id = s->next_id++;
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    *job = j->id;
  }
  s->cv_work.notify_one();
  return LC_OK;
}

extern "C" lc_status lc_server_cancel(lc_server* s, uint64_t job) {
  if (!s) return LC_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return LC_ERR_INVALID;
    Job* j = it->second;
    if (j->state == Job::kQueued) {
      auto q = std::find(s->queue.begin(), s->queue.end(), j);
      if (q != s->queue.end()) s->queue.erase(q);
      finish_job(s, j, LC_ERR_CANCELLED);
    } else if (j->state == Job::kRunning) {
      j->cancel = true;
    } else {
      return LC_ERR_INVALID;  // its labels are already being copied out, or it is done
    }
  }
  s->cv_work.notify_one();
  s->cv_done.notify_all();
  return LC_OK;
}

extern "C" lc_status lc_server_result(lc_server* s, uint64_t job, double timeout_s,
                                      uint32_t* rounds, double* latency_s, uint64_t* n_i,
                                      uint64_t* m_i, uint32_t cap) {
  if (!s) return LC_ERR_INVALID;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return LC_ERR_INVALID;
  Job* j = it->second;
  auto done = [j] { return j->state == Job::kDone; };
  if (timeout_s > 0) {
    if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), done))
      return LC_ERR_TIMEOUT;  // the job stays known: wait again later
  } else {
    s->cv_done.wait(lock, done);
  }
  if (rounds) *rounds = j->rounds;
  if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  lc_status st = j->status;
  if (st == LC_OK && (n_i || m_i)) {
    for (size_t i = 0; i < std::min<size_t>(cap, j->hn.size()); ++i) {
      if (n_i) n_i[i] = j->hn[i];
      if (m_i) m_i[i] = j->hm[i];
    }
    if (j->hn.size() > cap) st = LC_ERR_INVALID;
  }
  s->jobs.erase(it);
  delete j;
  return st;
}

extern "C" lc_status lc_server_wait(lc_server* s, uint64_t job, double timeout_s,
                                    uint32_t* rounds, double* latency_s) {
  return lc_server_result(s, job, timeout_s, rounds, latency_s, nullptr, nullptr, 0);
}

extern "C" lc_status lc_server_stats(lc_server* s, uint64_t* completed, uint64_t* peak_active,
                                     uint64_t* bytes_in_use) {
  if (!s) return LC_ERR_INVALID;
  std::lock_guard<std::mutex> lock(s->mu);
  if (completed) *completed = s->completed;
  if (peak_active) *peak_active = s->peak_active;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  return LC_OK;
}

extern "C" lc_status lc_server_destroy(lc_server* s) {
  if (!s) return LC_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->jobs) delete kv.second;
  for (auto c : s->pool) server_release(s, c);
  for (auto x : s->streams) {
    cudaStreamSynchronize(x);
    cudaStreamDestroy(x);
  }
  cudaMemPoolDestroy(s->mempool);
  for (auto p : s->pinned_chunks) cudaFreeHost(p);
  delete s;
  return LC_OK;
}
