/*
 * lc.h -- C ABI of the GB300 LocalContraction connected-components library.
 *
 * Method: "Connected Components at Scale via Local Contractions" (Lacki,
 * Mirrokni, Wlodarczyk; arXiv 1807.10727).  Each phase (Section 3) draws a fresh
 * random vertex ordering rho, maps every vertex to the minimum-rank vertex of
 * its closed neighbourhood N(v) (Section 2 defines N(v) to contain v), merges
 * the arborescences of that parent map, found by pointer jumping (Theorem
 * thm:tree-rounds), relabels, deduplicates and compacts the edges (the O(1)-round
 * contraction lemma; isolated nodes dropped as in Section 6, Empirical study), and repeats until
 * no edges remain (Section 3).  The per-phase maps are composed back down to the
 * input vertices (Section 6, Empirical study) and every vertex is labelled with the smallest
 * input id of its connected component.
 *
 * Conventions shared by every entry point:
 *  - Vertex ids are uint32 in [0, n); n <= 2^32 - 1.  Edges are undirected COO
 *    pairs (src[j], dst[j]), j < m, m <= 2^32 - 1; self-loops and duplicate
 *    edges are allowed and ignored by the result.
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are CPU memory (pinned memory gives full copy speed).
 *  - All GPU work is ordered on the CUDA stream given at creation (a
 *    cudaStream_t passed as void*; NULL = the legacy default stream).
 *    lc_run / lc_run_host return after the phase counters and labels have been
 *    produced on that stream and the counters copied to the host.
 *  - No call throws; every call returns an lc_status.  On an error the outputs
 *    are unspecified and the context stays usable unless the status is
 *    LC_ERR_CUDA (a CUDA runtime error, after which the context should be
 *    destroyed).
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef LC_H
#define LC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lc_ctx lc_ctx; /* opaque; owns all device scratch memory */

typedef enum {
  LC_OK = 0,
  LC_ERR_INVALID = 1,        /* bad argument, vertex id >= n, or output cap too small */
  LC_ERR_OOM = 2,            /* a device allocation failed */
  LC_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  LC_ERR_NO_CONVERGENCE = 4, /* more phases than the round cap (64 + 4*ceil(log2 n)) */
  LC_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
  LC_ERR_INTERNAL = 6,       /* an internal index check failed (corrupted state; the
                                offending access was skipped and reported on stderr) */
  LC_ERR_CANCELLED = 7       /* a server job was cancelled (lc_server_cancel) */
} lc_status;

typedef enum {
  LC_VARIANT_FOREST = 0,  /* closed-N parent, arborescences (default, Section 2/3) */
  LC_VARIANT_TWO_HOP = 1, /* label = min rank over N(N(v)) (Section 3, LocalContraction) */
  LC_VARIANT_TREE = 2     /* open-N parent, weakly connected components (TreeContraction) */
} lc_variant;

/* Create a context for one graph.
 *   n        number of vertices.
 *   d_src, d_dst  device uint32[m] edge endpoints, caller-owned, read-only for
 *            the lifetime of the context (never written).  Both NULL: the
 *            context allocates its own device input buffers of m edges, filled
 *            by lc_run_host.
 *   m        number of edges (may be 0).
 *   seed     seed of the phase orderings: phase i ranks vertex v of G_i by the
 *            high 32 bits of SplitMix64 (Steele, Lea, Flood 2014) output v+1 of
 *            the stream seeded with output i+1 of the stream seeded with seed;
 *            ties go to the smaller id (Section 3 asks for a uniformly random
 *            priority, redrawn every phase).
 *   stream   cudaStream_t as void*.
 *   out      receives the context.
 * Allocates all device scratch for a run (about 16*m + 40*n bytes plus sort
 * status words, and 64 MiB more for m >= 2^22: see "relabel_cache_slots");
 * returns LC_ERR_OOM if that fails.  Ids are validated on the
 * device during lc_run (LC_ERR_INVALID from lc_run). */
lc_status lc_create(uint32_t n, const uint32_t* d_src, const uint32_t* d_dst, uint64_t m,
                    uint64_t seed, void* stream, lc_ctx** out);

/* Select the phase variant (default LC_VARIANT_FOREST) and the small-graph
 * finish: once 0 < m_i <= finish_edges, that phase merges each connected
 * component of G_i into one node (the paper's single-machine union-find finish,
 * Section 6, Empirical study).  finish_edges = 0 (default) disables it.  Both change the phase
 * count and per-phase sizes, never the labels.
 *   LC_VARIANT_TWO_HOP  nodes are the classes of equal label l(v) = the
 *            min-key vertex of N(N(v)), each named by its label vertex (which
 *            need not belong to the class); allocates 8*n more device bytes
 *            on first selection (LC_ERR_OOM if that fails).
 *   LC_VARIANT_TREE     f(v) = min-key vertex of N(v) \ {v} (v itself when it
 *            has no other neighbour); nodes are the weakly connected
 *            components of f, named by the lower-key vertex of their terminal
 *            2-cycle (Lemmas lem:cycle and lem:wccs).
 * Returns LC_ERR_INVALID for an unknown variant, for finish_edges != 0 on a
 * batch context (lc_batch_create: the threshold is per graph), or while a run
 * of the context is in flight.  Contexts created by the serving loop and
 * lc_run_static always use the forest variant without finish. */
lc_status lc_configure(lc_ctx* ctx, lc_variant variant, uint64_t finish_edges);

/* MergeToLarge step (Section 5, the step of the O(log log n) analysis on
 * random graphs), off by default.  alpha: host uint32[count], copied; phase i
 * < count with alpha[i] > 0 ends with the step, with parameter alpha_i: a node
 * of the phase's contracted graph is large when at least alpha_i vertices of
 * G_i were merged into it, and its priority is the alpha_i-th largest phase-i
 * key (rank << 32 | id) among them; every node that is not large and has a
 * large node at distance 1 or 2 joins the large node of highest priority
 * (large nodes do not move).  The step is part of phase i: it changes
 * (n_{i+1}, m_{i+1}) and later phases, not the phase count's meaning nor the
 * labels.  It is skipped after a union-find finish phase.  count = 0 turns it
 * off.  Device scratch comes from the context's arena (about 40 bytes per
 * node of the contracted graph plus 12 per vertex of G_i).
 * Returns LC_ERR_INVALID for alpha == NULL with count > 0, for a batch
 * context, or while a run of the context is in flight. */
lc_status lc_set_merge_to_large(lc_ctx* ctx, const uint32_t* alpha, uint32_t count);

typedef enum {
  LC_DEDUP_HASH = 0, /* hashed bucket partition + per-bucket hash set (default) */
  LC_DEDUP_SORT = 1  /* full LSD radix sort of the edge keys, keep the first of each run */
} lc_dedup;

/* How each phase removes duplicate edges after relabelling (the "potential
 * duplicates are removed in a standard way" step of the O(1)-round
 * contraction lemma).  Both give the same edge set, hence the same labels,
 * phase count and per-phase sizes; they differ in speed and in the order of
 * the edges inside the context (sorted with LC_DEDUP_SORT, unspecified with
 * LC_DEDUP_HASH).  LC_DEDUP_HASH falls back to the sort for a phase whose
 * hash buckets overflow. */
lc_status lc_set_dedup(lc_ctx* ctx, lc_dedup mode);

/* Tuning parameters (no counterpart in the paper; they change speed only,
 * never results):
 *   "window_bytes"  L2 budget (bytes, >= 1 MiB) of one pass of the phase-0
 *                   closed-neighbourhood minimum: vertices are processed in
 *                   windows of window_bytes / 8 ids, one pass over the input
 *                   edges per window (default 192 MiB).
 *   "relabel_window_bytes"  when the phase-0 root array (4 bytes per vertex)
 *                   is larger than this, phase 0 relabels the input edges in
 *                   one pass per part of the array of at most this size (at
 *                   most 8 parts), each gathering roots from its part only
 *                   (default 160 MiB; needs n < 2^31).
 *   "relabel_cache_slots"  size (a power of two in [2^10, 2^26], or 0 = off)
 *                   of a device-wide direct-mapped cache of relabelled keys
 *                   used in phases with at least 2^22 edges: a key already in
 *                   it is dropped before the deduplication (in a filter pass
 *                   after the relabel with LC_DEDUP_HASH, inside the relabel
 *                   with LC_DEDUP_SORT), so repeated edges between the same
 *                   pair of nodes reach the deduplication a few times instead
 *                   of once per edge.  8 bytes per slot of device
 *                   memory, reallocated on change (default 2^23 for contexts
 *                   of at least 2^22 edges, else 0).  Not while a run is in
 *                   flight.
 *   "relabel_cache_admit"  a key missing from that cache enters it at one in
 *                   2^value of its occurrences (0..16, default 3), so that
 *                   keys seen once rarely evict repeated ones.
 *   "max_rounds"    phase cap (default 0: 64 + 4 log2 n, far above the
 *                   O(log n) bound); a run that needs more phases returns
 *                   LC_ERR_NO_CONVERGENCE.
 *   "spin_limit"    bound (1..2^30, default 2^24 polls) of each wait of a
 *                   partition pass on its predecessor tiles (decoupled
 *                   look-back); a wait that runs out ends the run with
 *                   LC_ERR_TIMEOUT, and the context stays usable.
 *   "inject_lookback_stall"  1: in the next partition pass, tile 0 publishes
 *                   nothing, so the waits behind it run out (a test of the
 *                   timeout path that faults nothing; one shot).
 *   "bucket_blocks" phase-0 edge grouping: 0 (default) = automatic (graphs of
 *                   at least "bucket_min_vertices" vertices, default 2^23),
 *                   1 = off, 2..32 = forced with that many vertex blocks.
 *                   The n ids are cut into near-equal blocks and the input
 *                   edges are copied, grouped by (lower block, higher block),
 *                   into a context buffer before phase 0's minimum and
 *                   relabel, so that both gather from two blocks of the
 *                   per-vertex arrays at a time, a slice that stays in L2.
 *   "bucket_window_bytes"  automatic block count: the smallest (>= 2) for
 *                   which two blocks of 8-byte minima fit this many bytes
 *                   (>= 1 MiB, default 64 MiB).
 *   "bucket_min_vertices"  see "bucket_blocks".
 *   "host_chunk_edges"  lc_run_host: edges per input copy (>= 1, default
 *                   2^25); see lc_run_host.
 *   "late_min_edges"  phases with at least this many edges (>= 1024, default
 *                   2^22) plan their deduplication after the relabel, below;
 *                   lowering it below the context's edge count allocates the
 *                   buffers those phases use.  Not while a run is in flight.
 *   "cache_in_relabel"  0 (default) / 1: in segmented phases, whether the
 *                   device-wide cache is probed by the relabel itself (the
 *                   filter pass then only sketches and scatters) instead of
 *                   by the filter pass.
 *   "seg_dedup"     1 (default) / 0: whether those phases deduplicate by
 *                   segments (below) or by the bucket partition.
 *   "jump_bits_min_vertices"  phases of at least this many vertices (default
 *                   2^23) and an average degree below 4 find the roots with
 *                   a bitmap of the roots (one bit per vertex, in L2) before
 *                   reading another vertex's parent pointer.
 *   "table_slots"   cap (a power of two >= 2^14, or 0 = none) on the table slots
 *                   the segmented deduplication uses; when the slices do not
 *                   fit at once they are processed in groups, and when one
 *                   slice does not fit the phase uses the bucket partition
 *                   (a test hook; default 0).
 *   "target_permille"  scale (1..10^6, default 1000) applied to the estimated
 *                   distinct-key count before sizing the tables or buckets
 *                   (a test hook: small values undersize them, which the
 *                   full-sort fallback then repairs).
 * Phases with at least "late_min_edges" edges size their deduplication from a
 * HyperLogLog estimate (Flajolet et al. 2007) of the distinct relabelled keys,
 * read back after a filter pass that drops keys found in the device-wide
 * cache; the others plan from m_i.  With "seg_dedup" those phases split the
 * keys into 256 segments by their top bits (the filter writes each kept key
 * into its segment's region) and keep the distinct keys of each segment with
 * an open-addressing table slice of about twice its estimated distinct keys
 * (a table of up to 2^28 slots, 8 bytes each, allocated with the other
 * buffers of these phases); segments are taken in order, so the slices in use
 * stay in L2.  A slice or bucket that overflows sends that phase to the full
 * sort (lc_dedup_fallbacks counts such phases).
 * Unknown names or out-of-range values give LC_ERR_INVALID. */
lc_status lc_set_param(lc_ctx* ctx, const char* name, uint64_t value);

/* Run the whole phase loop.
 *   d_labels  device uint32[n], caller-owned: labels[v] = smallest vertex id in
 *             v's connected component.
 *   rounds    host: number of phases R.  R = 0 exactly when m == 0; an input of
 *             self-loops only runs one phase.
 *   n_i, m_i  host uint64[cap]: vertices and edges of G_i for i < R (G_0 is the
 *             input as given, loops and duplicates counted in m_0).
 *   cap       length of n_i and m_i; R > cap gives LC_ERR_INVALID with *rounds
 *             set and the first cap entries filled.
 * Any of rounds / n_i / m_i may be NULL (then cap is ignored). */
lc_status lc_run(lc_ctx* ctx, uint32_t* d_labels, uint32_t* rounds, uint64_t* n_i, uint64_t* m_i,
                 uint32_t cap);

/* End-to-end variant for a context created with NULL edge pointers: copies the
 * host edge arrays h_src/h_dst (uint32[m]) to the device, runs the phase loop
 * and copies the labels to host h_labels (uint32[n]); other arguments as in
 * lc_run.  For a single graph whose phase 0 takes the closed-neighbourhood
 * minimum (forest and two-hop variants, no union-find finish in phase 0) the
 * copy overlaps phase 0: the edges go over in chunks of "host_chunk_edges"
 * on a second stream of the context, and each chunk, as soon as it has
 * arrived, is grouped by vertex-block pair and gets its share of the minimum
 * (Section 2's parent over N(v); a minimum of atomic updates, the same in any
 * order).  Beyond 256 chunks or 16384 (bucket, chunk) runs the chunks only
 * get phase 0's bucket counts and all edges are grouped once they are in.
 * The chunk-local grouping takes 132 KB of device memory per chunk and a
 * relabel tile list of 16 bytes per 4096 edges, allocated at the first such
 * call (LC_ERR_OOM if that fails).  The result is the one lc_run gives on the
 * same edges.  Pinned host buffers give full copy speed; pageable ones are
 * staged by the CUDA runtime. */
lc_status lc_run_host(lc_ctx* ctx, const uint32_t* h_src, const uint32_t* h_dst,
                      uint32_t* h_labels, uint32_t* rounds, uint64_t* n_i, uint64_t* m_i,
                      uint32_t cap);

/* Batched form: k independent graphs in one context, run together (each
 * phase's kernels cover every graph still holding edges), with results equal
 * to k separate lc_create/lc_run calls.
 *   h_n      host uint32[k]: vertices of graph g (local ids 0..h_n[g]-1).
 *   h_eoff   host uint64[k+1]: graph g's edges are d_src/d_dst[h_eoff[g],
 *            h_eoff[g+1]); h_eoff[0] = 0, non-decreasing.
 *   d_src, d_dst  device uint32[h_eoff[k]], local ids, caller-owned, read-only.
 *   h_seeds  host uint64[k]: rank seed of graph g (as lc_create's seed).
 * sum(h_n) and h_eoff[k] must be <= 2^32 - 1.  Local ids are validated during
 * lc_batch_run (LC_ERR_INVALID).  Destroy with lc_destroy. */
lc_status lc_batch_create(uint32_t k, const uint32_t* h_n, const uint64_t* h_eoff,
                          const uint32_t* d_src, const uint32_t* d_dst, const uint64_t* h_seeds,
                          void* stream, lc_ctx** out);

/* Run a batch context.
 *   d_labels  device uint32[sum h_n]: graph g's labels at offset
 *             sum_{h<g} h_n[h], local (smallest local id of the component).
 *   rounds    host uint32[k]: phases of graph g.
 *   n_i, m_i  host uint64[k * cap], graph-major: n_i[g * cap + i] is the
 *             vertex count of graph g's phase i, for i < min(rounds[g], cap).
 *   cap       phases stored per graph; a graph with more gives LC_ERR_INVALID
 *             after everything else has been filled.
 * Any of rounds / n_i / m_i may be NULL. */
lc_status lc_batch_run(lc_ctx* ctx, uint32_t* d_labels, uint32_t* rounds, uint64_t* n_i,
                       uint64_t* m_i, uint32_t cap);

/* Diagnostics of the last successful run, host uint64[cap] each (NULL to skip):
 * mp_i = edges of phase i left after relabelling and loop removal, before
 * deduplication (m'_i); emitted_i = how many of those the relabel step wrote
 * out (it skips repeats of a key it has just written, so the deduplication
 * reads fewer keys; emitted_i <= mp_i).  Returns the phase count in *rounds. */
lc_status lc_last_stats(const lc_ctx* ctx, uint32_t* rounds, uint64_t* mp_i, uint64_t* emitted_i,
                        uint32_t cap);

/* Deduplication of each phase of the last run (no counterpart in the paper;
 * used to count the bytes the deduplication must move), host arrays of cap
 * entries each (NULL to skip):
 *   kept_i    keys that reached the deduplication: emitted_i, less the
 *             repeats that the device-wide cache dropped in phases of at
 *             least 2^22 edges (see "relabel_cache_slots").
 *   passes_i  partition passes the hashed deduplication planned (0 for
 *             LC_DEDUP_SORT and for phases small enough for one bucket).
 * Returns the phase count in *rounds, and LC_ERR_INVALID if cap is smaller
 * than it (the first cap are filled). */
lc_status lc_last_dedup(const lc_ctx* ctx, uint32_t* rounds, uint64_t* kept_i, uint32_t* passes_i,
                        uint32_t cap);

/* Phases of all runs of the context so far whose hashed deduplication
 * overflowed a table slice or bucket set and was redone by the full sort (no
 * counterpart in the paper; the result is the same either way).  *count
 * receives the number. */
lc_status lc_dedup_fallbacks(const lc_ctx* ctx, uint64_t* count);

/* Per-kernel instrumentation (no counterpart in the paper; used to measure
 * the kernels against the HBM roofline).  Launch counts of every kernel are
 * always kept.  lc_profile(ctx, 1) additionally records a CUDA event pair
 * around every kernel launch on the context's stream and accumulates each
 * kernel's device time; lc_profile(ctx, 0) stops that.  Either call first
 * synchronises the stream and resets all counts and times to zero. */
lc_status lc_profile(lc_ctx* ctx, int on);

/* Counters of kernel k (k = 0, 1, ... until LC_ERR_INVALID): its name
 * (static string), launches and accumulated device milliseconds since the
 * last lc_profile call.  Any output pointer may be NULL. */
lc_status lc_kernel_stats(const lc_ctx* ctx, uint32_t k, const char** name, uint64_t* launches,
                          double* ms);

/* Release the context and all its device memory (stream-ordered frees after a
 * synchronisation of the context's stream).  NULL is accepted. */
lc_status lc_destroy(lc_ctx* ctx);

/* Serving: a request loop with continuous batching (no counterpart in the
 * paper; it runs many independent LocalContraction jobs on one GPU).
 * A worker thread admits submitted jobs in arrival order while a slot and the
 * device-memory budget allow, keeps each job's contracted graph on the device
 * between phases, and enqueues each job's next phase as soon as its previous
 * one completes, so phases of different jobs interleave and overlap on the
 * device (one CUDA stream per slot).  Idle contexts are kept and re-used for
 * later jobs of equal or smaller size.
 *   lc_server_create: budget_bytes = device bytes the server may hold
 *     (0: 80% of the free memory now); slots = jobs running at once (1..1024).
 *     Uses the current device.
 *   lc_server_submit: n, host h_src/h_dst uint32[m], seed as in lc_create;
 *     h_labels host uint32[n] receives the labels.  All three host arrays
 *     must stay valid until lc_server_wait returns (pinned memory lets the
 *     copies overlap).  *job receives an id.  LC_ERR_OOM if the job alone
 *     exceeds the budget.
 *   lc_server_wait: blocks until the job is done (or timeout_s seconds have
 *     passed, if timeout_s > 0: LC_ERR_TIMEOUT, the job stays pending);
 *     returns its status, its phase count and its latency (submission to
 *     labels on the host) in seconds; then forgets the job.
 *   lc_server_result: lc_server_wait that also fills host uint64[cap] n_i,
 *     m_i (either may be NULL) with the job's per-phase sizes, as lc_run does
 *     (LC_ERR_INVALID after filling cap of them if the job ran more phases).
 *   lc_server_cancel: a queued job is dropped at once; a running one stops
 *     at its next phase boundary, once the work it has on the device
 *     completes (its context is kept for later jobs).  Waiting on it then
 *     returns LC_ERR_CANCELLED.  LC_ERR_INVALID for an unknown job or one
 *     whose labels are already being copied out (it completes normally).
 *   lc_server_stats: jobs completed, the most jobs that ran at once, device
 *     bytes held.
 *   lc_server_destroy: finishes submitted jobs, then frees everything.
 * The contexts of a server take their device memory from a memory pool of the
 * server, stream-ordered on their slot's stream, and their pinned host
 * counters from blocks the server keeps, so that creating and releasing
 * contexts never waits on the device while other jobs run. */
typedef struct lc_server lc_server;
lc_status lc_server_create(uint64_t budget_bytes, uint32_t slots, lc_server** out);
lc_status lc_server_submit(lc_server* s, uint32_t n, const uint32_t* h_src, const uint32_t* h_dst,
                           uint64_t m, uint64_t seed, uint32_t* h_labels, uint64_t* job);
lc_status lc_server_wait(lc_server* s, uint64_t job, double timeout_s, uint32_t* rounds,
                         double* latency_s);
lc_status lc_server_result(lc_server* s, uint64_t job, double timeout_s, uint32_t* rounds,
                           double* latency_s, uint64_t* n_i, uint64_t* m_i, uint32_t cap);
lc_status lc_server_cancel(lc_server* s, uint64_t job);
lc_status lc_server_stats(lc_server* s, uint64_t* completed, uint64_t* peak_active,
                          uint64_t* bytes_in_use);
lc_status lc_server_destroy(lc_server* s);

/* Allocation-free connected components for small graphs.  (The paper has no
 * counterpart; this entry point serves callers that must not allocate device
 * memory: code running under another framework's allocator that already holds
 * the device memory, plug-ins or callbacks that may not touch the allocator,
 * and latency-critical loops that avoid cudaMalloc because it can synchronise
 * the device.)
 *
 * Same computation, outputs and errors as lc_create + lc_run + lc_destroy
 * with the default settings, for n <= LC_STATIC_MAX_N vertices and
 * m <= LC_STATIC_MAX_M edges.  Inputs (d_src, d_dst: device uint32[m]) and
 * outputs (d_labels: device uint32[n]; rounds, n_i, m_i: host, as in lc_run)
 * are the caller's.  All scratch lives in one static device array of
 * LC_STATIC_SCRATCH_BYTES bytes inside this library, which every GPU that loads
 * the library holds until the process exits; the call performs no device or
 * pinned-host allocation (cudaMalloc, cudaFree, cudaMallocHost or any
 * allocating library routine).
 *   - Larger n or m: LC_ERR_INVALID, before any device work.
 *   - The first call on a device looks up the array's device address with that
 *     device current (once per device); make that first call before any
 *     stream capture.
 *   - Like lc_run, the call blocks the host until the labels are on the
 *     device: it waits for the stream once per phase and copies the phase
 *     counters into host memory.
 *   - Every call on a device shares the array, which keeps the last call's
 *     contents (each call clears what it needs zeroed).  Calls whose GPU work
 *     overlaps (other streams, other host threads) race on it and give
 *     undefined results: serialise them.
 *   - Phase sequences that shrink very slowly can exceed the static per-phase
 *     storage (16 words per vertex): LC_ERR_OOM, labels not written. */
#define LC_STATIC_MAX_N 131072u
#define LC_STATIC_MAX_M 524288u
#define LC_STATIC_SCRATCH_BYTES (20u << 20)
lc_status lc_run_static(uint32_t n, const uint32_t* d_src, const uint32_t* d_dst, uint64_t m,
                        uint64_t seed, void* stream, uint32_t* d_labels, uint32_t* rounds,
                        uint64_t* n_i, uint64_t* m_i, uint32_t cap);

/* Test hook for the allocation-failure paths (no counterpart in the paper):
 * the k-th device or pinned-host allocation the library makes after this
 * call fails as if memory were exhausted (one shot; k = 0 turns the hook
 * off).  The pieces lc_run_static carves out of its static array count as
 * allocations here (it still calls no allocator).  The call that made it returns LC_ERR_OOM and releases what it had
 * allocated; the library stays usable.  Process-wide. */
lc_status lc_fail_alloc(uint64_t k);

/* Static text for a status code. */
const char* lc_status_str(lc_status s);

/* Phase ordering rank, for parity checks: the 32-bit rank of vertex v in phase
 * i, computed on the device by the same code the phases use.  d_out is device
 * uint32[count] receiving rank(seed, i, v0 + j) for j < count. */
lc_status lc_rank_probe(uint64_t seed, uint32_t i, uint32_t v0, uint32_t count, uint32_t* d_out,
                        void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LC_H */
