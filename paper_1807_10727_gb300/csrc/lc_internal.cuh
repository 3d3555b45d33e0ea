// Host-side launchers of the LocalContraction kernels (internal to liblc.so).
#pragma once
#include <cstdint>
#include <tuple>
#include <vector>
#include <cuda_runtime.h>

#include "lc_common.cuh"

namespace lc {

// Every kernel of the library, for launch counting and per-kernel timing.
enum KernelId : int {
  kKInitKeys,
  kKEdgeMinSoa,
  kKEdgeMinPacked,
  kKJump,
  kKRelabelSoa,
  kKRelabelPacked,
  kKRelabelSplit,
  kKSortHist,
  kKHistScan,
  kKSortPass,
  kKScanFlags,
  kKUniqueRename,
  kKPropagate,
  kKBucketBounds,
  kKBucketDedup,
  kKRename,
  kKUnmix,
  kKBatch,
  kKTwoHop,
  kKOpenMin,
  kKTreeNames,
  kKUnionFind,
  kKMergeGroup,
  kKMergeSelect,
  kKMergeHop,
  kKMergeTarget,
  kKIdentity,
  kKRankProbe,
  kKFilter,
  kKBucketEdges,
  kKSegDedup,
  kNumKernels
};

const char* kernel_name(int id);

// Launch counts (always) and, when `on`, device time of every launch measured
// with a CUDA event pair recorded around it on the launching stream.
struct Prof {
  bool on = false;
  uint64_t launches[kNumKernels] = {};
  double ms[kNumKernels] = {};
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void resolve();  // call after the stream has been synchronised
  void reset();
  void release();
};

struct Launch {
  cudaStream_t stream;
  int sms;             // multiprocessor count of the device
  Prof* prof = nullptr;
};

// Scope around one kernel launch: counts it and, when timing is on, brackets
// it with events.
struct KScope {
  const Launch& L;
  int id;
  cudaEvent_t e0 = nullptr;
  KScope(const Launch& l, int k) : L(l), id(k) {
    if (L.prof) {
      ++L.prof->launches[k];
      if (L.prof->on) {
        e0 = L.prof->get();
        cudaEventRecord(e0, L.stream);
      }
    }
  }
  ~KScope() {
    if (e0) {
      cudaEvent_t e1 = L.prof->get();
      cudaEventRecord(e1, L.stream);
      L.prof->pending.emplace_back(id, e0, e1);
    }
  }
};

// ---------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per tile
constexpr int kRadixBits = 8;        // digit width of the full-key sort
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRadixBitsMax = 8;     // widest digit of a hashed partition pass
constexpr int kRadixMax = 1 << kRadixBitsMax;
static_assert(kRadixMax % 256 == 0, "scan kernels assume whole digits per thread");
constexpr int kMaxPasses = 8;
constexpr int kBucketTarget = 2048;  // average keys per dedup bucket
constexpr int kMaxHashBits = 24;
constexpr int kHllBits = 11;                 // HyperLogLog: 2^11 registers
constexpr int kHllRegs = 1 << kHllBits;

// Digit of a key in one pass: bits [shift, shift + bits).
struct DigitFn {
  int shift;
  uint32_t mask;
  __device__ __forceinline__ uint32_t operator()(uint64_t k) const {
    return (uint32_t)(k >> shift) & mask;
  }
};

// The digits of an LSD sort or partition, least significant pass first.
struct PassPlan {
  int passes;
  int shift[kMaxPasses];
  int bits[kMaxPasses];
  __host__ __device__ DigitFn digit_fn(int p) const {
    return DigitFn{shift[p], (1u << bits[p]) - 1u};
  }
  __device__ __forceinline__ uint32_t digit(int p, uint64_t k) const {
    return (uint32_t)(k >> shift[p]) & ((1u << bits[p]) - 1u);
  }
};

// Scratch of the onesweep sort and the single-pass scans.  `status` holds one
// 64-bit look-back word per (tile, digit); epochs make stale words invalid so
// the array never needs clearing between launches.
struct SortScratch {
  uint64_t* status = nullptr;     // [status_words]
  uint64_t status_words = 0;
  uint32_t* hist = nullptr;       // [kMaxPasses * kRadixMax] global digit counts / offsets
  unsigned* tickets = nullptr;    // [16] dynamic tile counters
  uint32_t epoch = 0;             // last epoch used (1..2^30-1)
  uint32_t spin_limit = kSpinLimit;  // bound of each partition-pass look-back wait
  int stall_once = 0;             // test hook: the next partition pass's tile 0 stays silent
};

uint64_t sort_status_words(uint64_t max_keys);

// Next epoch for a look-back launch; clears the status array when the epoch
// counter wraps.
uint32_t next_epoch(SortScratch& s, const Launch& L);

// Stable LSD radix sort of keys[0, *d_count) on bits [0, key_bits) with 8-bit
// digits (onesweep: one histogram pass, then one single-pass scatter per digit
// with decoupled look-back).  `max_count` bounds *d_count and sizes the grids.
// The sorted keys end in keys or alt; the return value says which (0 = keys).
// When mark_flags is non-null the last pass also sets the bits of a and b in
// the mark_flags bitmap for every key (a << half_bits | b) (used to find the
// nodes that keep an edge).
int radix_sort_u64(uint64_t* keys, uint64_t* alt, const unsigned long long* d_count,
                   uint64_t max_count, int key_bits, SortScratch& s, unsigned* err,
                   uint32_t* mark_flags, int half_bits, const Launch& L);

// Bucket-hash bits used for max_count keys (0 when one bucket suffices).
int hash_bits_for(uint64_t max_count);

// Partition plan over the top hb = hash_bits_for(max_count) bits of the mixed
// keys (digits of at most kRadixBitsMax bits, two passes up to 18 bits).
// Returns hb.
int hash_plan(uint64_t max_count, PassPlan* plan);

// Zero the digit counts of s.hist (before a producer accumulates them).
void hist_reset(SortScratch& s, const Launch& L);

// ------------------------------------------------- phase-0 edge buckets
// The n vertex ids are cut into nb near-equal blocks (block of v =
// min(umulhi(v, scale), nb - 1)); an edge belongs to the bucket (lower block,
// higher block), numbered lo * nb + hi.  Grouping the input edges by bucket
// (ascending bucket number, rows of one lower block together) means that, at
// any moment, the edges in flight gather per-vertex data from about two
// blocks, a slice of the vertex arrays that stays in L2.
constexpr uint32_t kBucketMaxBlocks = 32;
constexpr uint32_t kBucketMaxDigits = kBucketMaxBlocks * kBucketMaxBlocks;
constexpr uint32_t kBucketFillStride = 32;  // words between fill counters (one line each)
// scratch words: counts [0, kBucketMaxDigits), padded fill counters, then the
// segment starts and tile prefixes of the segmented deduplication (below)
constexpr uint64_t kSegStartOff = kBucketMaxDigits * (1 + kBucketFillStride);
constexpr uint64_t kSegTileOff = kSegStartOff + 512;
constexpr uint64_t kBucketScratchWords = kSegTileOff + 512;

// Blocks used for n vertices so that two blocks of 8-byte per-vertex data
// fit in window_bytes (at least 2, at most kBucketMaxBlocks).
uint32_t bucket_blocks_for(uint32_t n, uint64_t window_bytes);

// out[0, m) = the input edges (u << 32 | v) grouped by bucket (order inside a
// bucket unspecified).  Ids >= n set kErrBadVertex and become the self-loop
// (0, 0), which no step counts.  scratch: kBucketScratchWords words.
// bucket_edges = bucket_clear, then bucket_count over all edges (which may be
// split into several calls on consecutive parts), then bucket_place.
void bucket_clear(uint32_t n, uint32_t nb, uint32_t* scratch, const Launch& L);
void bucket_count(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t nb,
                  uint32_t* scratch, unsigned* err, const Launch& L);
void bucket_place(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t nb,
                  uint64_t* out, uint32_t* scratch, unsigned* err, const Launch& L);
void bucket_edges(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t nb,
                  uint64_t* out, uint32_t* scratch, unsigned* err, const Launch& L);

// Chunk-local grouping (lc_run_host): chunk c = edges [c * chunk, ...) is
// grouped on its own into out[c * chunk, ...) with bucket_edges, using
// chunk_scratch + c * kChunkScratchWords; chunk_tiles then lists, in bucket
// order and chunk order inside a bucket, tiles of at most tile_edges edges
// that never cross a (bucket, chunk) run: tiles[2t] = first edge, tiles[2t+1]
// = end; *ntiles = their number.  `tiles` holds chunk_tiles_bytes(...) bytes;
// the launch scans nb^2 * chunks segments in one block (keep that small).
constexpr uint64_t kChunkScratchWords = (uint64_t)kBucketMaxDigits * (1 + kBucketFillStride);
constexpr uint32_t kRelabelTileEdges = 4096;  // edges per relabel tile (kernel constant)
uint64_t chunk_tiles_bytes(uint64_t m, uint32_t nb, uint32_t chunks, uint32_t tile_edges);
void chunk_tiles(const uint32_t* chunk_scratch, uint32_t chunks, uint64_t chunk, uint64_t m,
                 uint32_t n, uint32_t nb, uint32_t tile_edges, uint64_t* tiles,
                 unsigned long long* ntiles, unsigned* err, const Launch& L);

// -------------------------------------------- segmented deduplication
// Large phases: the relabel counts its (mixed) keys per segment, the top
// kSegBits bits, into scratch[0, kSegs); seg_begin turns the counts into
// segment regions; filter_seg drops repeats (device-wide cache, as
// filter_hll) and writes every kept key into its segment's region; seg_dedup
// then keeps the distinct keys of each segment with an open-addressing table
// slice of `slots` entries per segment, taking the segments in order so that
// the slices in use stay in L2.  seg_compact copies the kept keys of all
// segments into one contiguous array (before a full-sort fallback).
constexpr int kSegBits = 8;
constexpr uint32_t kSegs = 1u << kSegBits;

void seg_begin(uint32_t* scratch, const Launch& L);
void filter_seg(const uint64_t* in, const unsigned long long* d_in, uint64_t max_count,
                uint64_t* out, unsigned long long* d_out, unsigned long long* gcache,
                uint32_t gslots, int admit, uint32_t* hll, uint32_t* scratch, unsigned* err,
                const Launch& L);
// Returns false when the table cannot hold kSegs slices of `slots` entries
// (the caller then compacts and uses hash_dedup).  Overflow of a slice sets
// kErrOverflow (the caller falls back to the full sort).
bool seg_dedup(const uint64_t* keys, uint32_t* scratch, uint64_t max_count, uint64_t* table,
               uint64_t table_slots, uint64_t slots, uint64_t* out, unsigned long long* m_next,
               uint32_t* flags, uint32_t n, int half_bits, unsigned* ticket, unsigned* err,
               const Launch& L);
void seg_compact(const uint64_t* keys, const uint32_t* scratch, uint64_t* out, const Launch& L);

// Duplicate filter and distinct-count sketch of the *d_in mixed keys in `in`:
// keys found in the device-wide cache (gcache, gslots slots, a power of two,
// ~0 in every slot when a phase starts using it; 0 slots = keep all) are
// dropped, the others appended to out (count added to *d_out, zero before)
// and entered in the cache at one in 2^admit of their positions; hll
// (kHllRegs words, zero before) receives the HyperLogLog registers (Flajolet
// et al. 2007) of the kept keys.  The kept keys hold every distinct key.
void filter_hll(const uint64_t* in, const unsigned long long* d_in, uint64_t max_count,
                uint64_t* out, unsigned long long* d_out, unsigned long long* gcache,
                uint32_t gslots, int admit, uint32_t* hll, const Launch& L);

// Duplicate removal without a full sort, on mixed keys (key_mix of
// a << half_bits | b): a stable LSD partition of keys[0, *d_count) by their
// top hb bits following `plan` (from hash_plan; with hist_ready the digit
// counts are already in s.hist), so all copies
// of a key share one bucket of about kBucketTarget keys; then one block per
// bucket keeps the distinct keys with a shared-memory hash set, appends them
// (mixed, in no particular order) to the other buffer, counts them in *m_next
// and marks both endpoints in flags.  Returns
// which buffer holds the partitioned keys (0 = keys, 1 = alt); the distinct
// keys are in the other one.  A bucket whose distinct keys overflow the set
// raises kErrOverflow (the caller then falls back to radix_sort_u64).
// `bounds` holds (1 << hb) + 1 words.
int hash_dedup(uint64_t* keys, uint64_t* alt, const unsigned long long* d_count,
               uint64_t max_count, const PassPlan& plan, int hb, bool hist_ready,
               int half_bits, uint32_t* flags, uint32_t n, uint32_t* bounds,
               unsigned long long* m_next, SortScratch& s, unsigned* err, const Launch& L);

// e[j] = (id(a) << 32 | id(b)) for each mixed key e[j] = key_mix(a <<
// half_bits | b), j < *d_count, with id the keep rank (keep_rank).
void rename_edges(uint64_t* e, const unsigned long long* d_count, uint64_t max_count,
                  int half_bits, const uint64_t* rank, uint32_t n, unsigned* err,
                  const Launch& L);

// In place: e[j] = key_unmix(e[j]) for j < *d_count.
void unmix_keys(uint64_t* e, const unsigned long long* d_count, uint64_t max_count,
                const Launch& L);

// Keep ranks rank[0, rank_words(n)) of the flag bits 0..n-1 (bitmap, see
// flag_words): an exclusive scan of the words' popcounts; for every kept r
// (flag set) also copies mo_in[r] to mo_out[id(r)] when mo_out is non-null.
// *total gets the number of kept nodes.
void scan_flags(const uint32_t* flags, uint64_t* rank, uint32_t n, const uint32_t* mo_in,
                uint32_t* mo_out, unsigned long long* total, SortScratch& s, unsigned* err,
                const Launch& L);

// Compaction of the sorted keys[0, *d_count): keeps the first key of each run
// of equal keys and writes it renamed through the keep ranks as (id(a) << 32
// | id(b)) to out in sorted order; *m_next gets the number kept.
void unique_rename(const uint64_t* keys, const unsigned long long* d_count, uint64_t max_count,
                   int half_bits, const uint64_t* rank, uint32_t n, uint64_t* out,
                   unsigned long long* m_next, SortScratch& s, unsigned* err, const Launch& L);

// ---------------------------------------------------------- phase steps
// A batch of independent graphs in one id space (device pointers): graph g
// owns ids [voff[g], voff[g+1]) and uses phase seed rk[g], passed as
// gs[g] = rk[g] + (1 - voff[g]) * kGamma (batch_phase_seeds).
struct BatchView {
  const uint64_t* gs;
  const uint32_t* voff;
  uint32_t k;
  const uint32_t* gid;  // graph of every vertex of the level (batch_graph_ids)
};

// minkey[v] = key(v) for v < n; when mo is non-null also mo[v] = v (phase 0).
// With a batch, each vertex is keyed by its own graph's seed and local id.
void init_keys(unsigned long long* minkey, uint32_t* mo, uint32_t n, uint64_t rk,
               const BatchView* batch, const Launch& L);

// Closed-neighbourhood minimum: minkey[u] = min(minkey[u], key(v)) and
// minkey[v] = min(minkey[v], key(u)) for every edge.  Edges are either two
// uint32 arrays (src, dst) with ids validated against n (bad ids set
// kErrBadVertex and are skipped), or packed uint64 (a << 32 | b) sorted by a
// (packed != nullptr).  For the uint32 form, vertices are processed in windows
// of at most window_bytes / 8 ids, one pass over the edges per window, so that
// each pass's atomics stay inside an L2-sized slice of minkey.  open: the
// open-neighbourhood minimum (no vertex offers its own key; the caller fills
// minkey with ~0 first), two atomics per edge.
void edge_min(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
              uint32_t n, uint64_t rk, unsigned long long* minkey, unsigned* err,
              uint64_t window_bytes, const BatchView* batch, const Launch& L, bool open = false);

// Batches: phase seeds gs[g] for phase i (see BatchView); local -> global edge ids (ids
// validated per graph); next level offsets voff_next[g] = id(voff[g]) (keep
// ranks of the level), the next level's graph ids gid[0, n_next) and the
// per-graph edge counts of its packed edges e[0, m); global -> local labels.
void batch_phase_seeds(const uint64_t* seeds, uint32_t k, uint32_t i, const uint32_t* voff,
                       uint64_t* gs, const Launch& L);
void batch_globalize(const uint32_t* src, const uint32_t* dst, const uint64_t* eoff,
                     const uint32_t* voff, uint32_t k, uint64_t m, uint32_t* gsrc, uint32_t* gdst,
                     unsigned* err, const Launch& L);
void batch_next_level(const uint32_t* voff, const uint64_t* rank, uint32_t k, uint32_t* voff_next,
                      const uint64_t* e, uint64_t m, uint32_t* mcnt, uint32_t n_next,
                      uint32_t* gid, const Launch& L);
// gid[v] = graph of vertex v, v < n = voff[k].
void batch_graph_ids(const uint32_t* voff, uint32_t k, uint32_t n, uint32_t* gid,
                     const Launch& L);
void batch_localize(uint32_t* labels, uint32_t n, const uint32_t* voff, uint32_t k,
                    const Launch& L);

// root[v] = root of v's arborescence (follows the parent stored in the low
// half of minkey, compressing as it goes); mo[root] = min over the tree of
// mo[v] (phase 0: mo[v] = v).  isroot: flag_words(n) words of scratch, which
// receive a bitmap of the roots when the phase (n vertices, m edges) has at
// least bits_min_vertices vertices and an average degree below 4.
// A chase longer than n steps (only possible with corrupted data) stops and
// records the failed index check.
void jump(unsigned long long* minkey, uint32_t* root, uint32_t* mo, uint32_t n, uint64_t m,
          uint32_t* isroot, uint32_t bits_min_vertices, unsigned* err, const Launch& L);

// Relabel every edge through root, drop self-loops, emit (min << bits | max)
// keys (mixed with key_mix when `mix`) compacted to keys_out.  With `plan`
// non-null the digit counts of the written keys under that plan are added to
// ghist (the partition histogram, so the dedup needs no extra read).  For
// uint32 input with n * 4 > window_bytes (and n < 2^31) the relabel runs in
// two passes, each gathering from one L2-sized half of root, with `tmp`
// (8 bytes per edge) holding the half-resolved edges in between.  *mprime gets the number of non-loop edges;
// *emitted the number of keys written, which omits repeats of a key that the
// same block has already written or that the device-wide cache holds (gcache:
// gslots 64-bit slots, a power of two, all ~0 when the phase's relabel
// starts; nullptr / 0 = no such cache; a missing key enters it at one in
// 2^admit of its occurrences).  The written keys hold every distinct key.
// Tiles are claimed in order through the device word `ticket` (cleared here).
// Packed edges may come with a tile list (tiles, *d_ntiles: see chunk_tiles),
// which then replaces the tiles of consecutive edges.
void relabel(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
             uint32_t n, const uint32_t* root, int bits, uint64_t* keys_out,
             unsigned long long* mprime, unsigned long long* emitted, bool mix,
             const PassPlan* plan, uint32_t* ghist, uint64_t* tmp, uint64_t window_bytes,
             unsigned long long* gcache, uint32_t gslots, int admit, unsigned* ticket,
             unsigned* err, const Launch& L, const uint64_t* tiles = nullptr,
             const unsigned long long* d_ntiles = nullptr);

// labels_out[v] = kept(root[v]) ? labels_up[id(root[v])] : mo[root[v]], with
// kept and id from the level's keep ranks.  labels_out may alias root.
void propagate(const uint32_t* root, const uint64_t* rank, const uint32_t* mo,
               const uint32_t* labels_up, uint32_t* labels_out, uint32_t n, uint32_t n_up,
               unsigned* err, const Launch& L);

// ctr->tag = tag, ordered after everything enqueued before it on the stream
// (lets the host check that the counters it reads belong to the phase it
// expects).
void stamp_counters(Counters* ctr, uint64_t tag, const Launch& L);

// Node names of the other phase variants (edges as in edge_min; root[v]
// receives the name of v's node):
//  - two_hop_names: published LocalContraction label, min key over N(N(v))
//    (mk1 = closed-neighbourhood minima from edge_min; mk2 and fpar, n words,
//    scratch; rk / batch give the keys); names need not be members of their
//    group, so node minima go to nmo (n words).
//  - tree_names: TreeContraction, parent = low half of the open-neighbourhood
//    minimum in minkey (edge_min with open; ~0 = no other neighbour), name =
//    lower-key vertex of the terminal 2-cycle; node minima in mo in place.
//  - union_find_names: every vertex named by its component's smallest id
//    (the small-graph finish); parent is n words of scratch.
void two_hop_names(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
                   uint32_t n, uint64_t rk, const BatchView* batch,
                   const unsigned long long* mk1, unsigned long long* mk2, uint32_t* fpar,
                   uint32_t* root, const uint32_t* mo, uint32_t* nmo, unsigned* err,
                   const Launch& L);
void tree_names(const unsigned long long* minkey, uint32_t* root, uint32_t* mo, uint32_t n,
                uint64_t rk, const BatchView* batch, unsigned* err, const Launch& L);
void union_find_names(const uint32_t* src, const uint32_t* dst, const uint64_t* packed,
                      uint64_t m, uint32_t n, uint32_t* parent, uint32_t* root, uint32_t* mo,
                      unsigned* err, const Launch& L);

// Scratch of the MergeToLarge step: n' words for cnt, off, fill, list and
// n' 64-bit words for prio, h1, h2 (n' = nodes of the contracted graph); n_i
// words for members and n_i 64-bit words for cand (n_i = vertices of the
// phase's input); three counter words; the big-node tables.
struct MergeScratch {
  uint32_t *cnt, *off, *fill, *list, *members;
  unsigned long long *cand, *prio, *h1, *h2;
  unsigned* ctrs;  // 3 words
  uint32_t* big;   // merge_big_words(n_i) words: nodes of >= 2^15 members
};

// Words of MergeScratch::big for a phase input of n_i vertices.
inline uint64_t merge_big_words(uint32_t n_i) {
  const uint64_t nb = n_i / (1u << 15) + 1;
  return nb * (1 + 256 + 1) + 1 + 2 * nb;
}

// MergeToLarge (Section 5) on the graph G' (n2 nodes, packed edges e[m])
// that the last phase made from G_i (n_i vertices; root_i, rank_i its root
// map and keep ranks; rk its key seed): t[x] = node that x joins (x itself
// when it stays); node minima mo aggregated in place at the targets.
void merge_to_large_names(const uint32_t* root_i, const uint64_t* rank_i, uint32_t n_i,
                          uint64_t rk, uint32_t alpha, const uint64_t* e, uint64_t m,
                          uint32_t n2, uint32_t* t, uint32_t* mo, const MergeScratch& s,
                          unsigned* err, const Launch& L);

// labels[v] = v (a graph without edges).
void identity_labels(uint32_t* labels, uint32_t n, const Launch& L);

// out[j] = high 32 bits of key(v0 + j) in the phase with stream seed rk.
void rank_probe(uint64_t rk, uint32_t v0, uint32_t count, uint32_t* out, const Launch& L);

}  // namespace lc
