// Per-phase kernels of the LocalContraction round loop (arXiv 1807.10727):
// ranking and closed-neighbourhood parent (Section 2 N(v), Section 3 random
// ordering), contraction of the parent arborescences by pointer jumping
// (Theorem thm:tree-rounds), relabelling of the edges (O(1)-round contraction
// lemma) and composition of the per-phase maps back to the input (Section 6, Empirical study).
#include <algorithm>

#include "lc_internal.cuh"

namespace lc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 256;

inline int grid_for(uint64_t work, int per_block, const Launch& L, int blocks_per_sm = 8) {
  uint64_t b = (work + per_block - 1) / per_block;
  uint64_t cap = (uint64_t)L.sms * blocks_per_sm;
  return (int)std::max<uint64_t>(1, std::min(b, cap));
}

// ------------------------------------------------------------ ranking

// Keys of one phase of a single graph: the phase's stream seed and the id.
struct GraphKeys {
  uint64_t rk;
  __device__ __forceinline__ uint64_t key(uint32_t v) const { return phase_key(rk, v); }
  __device__ __forceinline__ void pair(uint32_t u, uint32_t v, uint64_t& ku, uint64_t& kv) const {
    ku = phase_key(rk, u);
    kv = phase_key(rk, v);
  }
};

// Keys of one phase of a batch of independent graphs sharing one id space:
// graph g owns ids [voff[g], voff[g+1]) and ranks its vertex v with its own
// phase seed rk[g] and its local id v - voff[g], exactly as a run on graph g
// alone would.  The low half keeps the global id (the order inside a graph is
// the same) so that it can index the per-vertex arrays.  Edges never cross
// graphs, so both endpoints of an edge share one lookup.
struct BatchKeys {
  const uint64_t* gs;  // per graph: phase seed rk[g] + (1 - voff[g]) * kGamma (mod 2^64)
  const uint32_t* voff;
  uint32_t k;
  const uint32_t* gid = nullptr;  // graph of every vertex of the level (nullptr: search voff)
  __device__ __forceinline__ uint32_t graph_of(uint32_t v) const {
    if (gid != nullptr) return __ldg(gid + v);
    uint32_t lo = 0, hi = k - 1;  // last g with voff[g] <= v
    while (lo < hi) {
      uint32_t mid = (lo + hi + 1) >> 1;
      if (__ldg(voff + mid) <= v) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
  // rk[g] + (v - voff[g] + 1) * kGamma, the stream input of local id
  // v - voff[g], equals gs[g] + v * kGamma: one per-graph word per key
  __device__ __forceinline__ uint64_t key_in(uint32_t g, uint32_t v) const {
    return (splitmix_mix(__ldg(gs + g) + (uint64_t)v * kGamma) & 0xFFFFFFFF00000000ull) | v;
  }
  __device__ __forceinline__ uint64_t key(uint32_t v) const { return key_in(graph_of(v), v); }
  __device__ __forceinline__ void pair(uint32_t u, uint32_t v, uint64_t& ku, uint64_t& kv) const {
    const uint32_t g = graph_of(u);
    ku = key_in(g, u);
    kv = key_in(g, v);
  }
};

template <class K>
__global__ void k_init_keys(unsigned long long* __restrict__ minkey, uint32_t* __restrict__ mo,
                            uint32_t n, K keys) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    minkey[v] = keys.key((uint32_t)v);
    if (mo != nullptr) mo[v] = (uint32_t)v;
  }
}

__global__ void k_rank_probe(uint64_t rk, uint32_t v0, uint32_t count, uint32_t* out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride)
    out[j] = (uint32_t)(phase_key(rk, (uint32_t)(v0 + j)) >> 32);
}

// ---------------------------------------------------- closed-N minimum

// Window form of the edge update: keys are distinct, so of key(u) and key(v)
// only the larger endpoint's minimum can drop, to the other endpoint's key;
// the edge needs one atomic, applied when that endpoint lies in
// [lo, lo + span) (so one pass over the edges touches an L2-sized slice of
// minkey).  kOpen: the open-neighbourhood minimum of TreeContraction (minkey
// starts at ~0, not at the vertex's own key), where both endpoints take the
// other's key, each when it lies in the window.
template <bool kOpen, class K>
__device__ __forceinline__ void min_edge_window(uint32_t u, uint32_t v, uint32_t n, const K& keys,
                                                unsigned long long* minkey, unsigned* err,
                                                uint32_t lo, uint32_t span, bool check) {
  if (check && (u >= n || v >= n)) {
    atomicOr(err, kErrBadVertex);
    return;
  }
  if (u == v) return;
  uint64_t ku, kv;
  keys.pair(u, v, ku, kv);
  if (kOpen) {
    if (u - lo < span) min_if_lower(&minkey[u], (unsigned long long)kv);
    if (v - lo < span) min_if_lower(&minkey[v], (unsigned long long)ku);
    return;
  }
  const uint32_t hi = ku < kv ? v : u;
  if (hi - lo < span) min_if_lower(&minkey[hi], (unsigned long long)(ku < kv ? ku : kv));
}

// Input edges as two uint32 arrays; `vec` = both arrays 16-byte aligned.
// Updates only vertices in [lo, lo + span); ids are validated when `check`.
template <bool kOpen, class K>
__global__ void __launch_bounds__(kThreads) k_edge_min_soa(
    const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m, uint32_t n,
    K keys, unsigned long long* minkey, unsigned* err, int vec, uint32_t lo, uint32_t span,
    int check) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t done = 0;
  if (vec) {
    const uint64_t nq = m / 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const uint4* d4 = reinterpret_cast<const uint4*>(dst);
    for (uint64_t q = gt; q < nq; q += stride) {
      uint4 s = __ldcs(s4 + q), d = __ldcs(d4 + q);
      min_edge_window<kOpen>(s.x, d.x, n, keys, minkey, err, lo, span, check);
      min_edge_window<kOpen>(s.y, d.y, n, keys, minkey, err, lo, span, check);
      min_edge_window<kOpen>(s.z, d.z, n, keys, minkey, err, lo, span, check);
      min_edge_window<kOpen>(s.w, d.w, n, keys, minkey, err, lo, span, check);
    }
    done = nq * 4;
  }
  for (uint64_t j = done + gt; j < m; j += stride)
    min_edge_window<kOpen>(__ldcs(src + j), __ldcs(dst + j), n, keys, minkey, err, lo, span,
                           check);
}

// One atomic per edge, at the endpoint with the larger key (see
// min_edge_window); two for the open-neighbourhood minimum.
template <bool kOpen, class K>
__device__ __forceinline__ void min_edge_packed(uint64_t x, const K& keys,
                                                unsigned long long* minkey, uint32_t n,
                                                unsigned* err) {
  const uint32_t a = (uint32_t)(x >> 32), b = (uint32_t)x;
  if (!index_ok(err, kOpen ? kKOpenMin : kKEdgeMinPacked, max(a, b), n)) return;
  // a self-loop (phase 0's grouped input keeps them) offers no other
  // neighbour: it must not reach the open-neighbourhood minimum
  if (kOpen && a == b) return;
  uint64_t ka, kb;
  keys.pair(a, b, ka, kb);
  if (kOpen) {
    min_if_lower(&minkey[a], (unsigned long long)kb);
    min_if_lower(&minkey[b], (unsigned long long)ka);
  } else if (ka < kb) {
    min_if_lower(&minkey[b], (unsigned long long)ka);
  } else {
    min_if_lower(&minkey[a], (unsigned long long)kb);
  }
}

// Packed edges (a << 32 | b), two per 128-bit load.
template <bool kOpen, class K>
__global__ void __launch_bounds__(kThreads) k_edge_min_packed(
    const uint64_t* __restrict__ e, uint64_t m, K keys, unsigned long long* minkey, uint32_t n,
    unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t npair = m / 2;
  const ulonglong2* e2 = reinterpret_cast<const ulonglong2*>(e);
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t q = gt; q < npair; q += stride) {
    ulonglong2 p = __ldcs(e2 + q);
    min_edge_packed<kOpen>(p.x, keys, minkey, n, err);
    min_edge_packed<kOpen>(p.y, keys, minkey, n, err);
  }
  if ((m & 1) && gt == 0) min_edge_packed<kOpen>(e[m - 1], keys, minkey, n, err);
}

// ------------------------------------------------------- batches

// gs[g] = rk[g] + (1 - voff[g]) * kGamma, with rk[g] the stream seed of
// phase i for graph g (see BatchKeys).
__global__ void k_batch_phase_seeds(const uint64_t* __restrict__ seeds, uint32_t k, uint32_t i,
                                    const uint32_t* __restrict__ voff, uint64_t* __restrict__ gs) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < k; g += gridDim.x * blockDim.x)
    gs[g] = splitmix_mix(seeds[g] + (uint64_t)(i + 1) * kGamma) + kGamma -
            (uint64_t)voff[g] * kGamma;
}

// Last g with off[g] <= x in a non-decreasing offset array off[0..k].
template <class T>
__device__ __forceinline__ uint32_t segment_of(const T* __restrict__ off, uint32_t k, uint64_t x) {
  uint32_t lo = 0, hi = k - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if ((uint64_t)__ldg(off + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Work split of the batch kernels that walk a range in offset order: warp w
// takes items [w * chunk, (w + 1) * chunk) (chunk a multiple of 32), four
// per lane per step; lane 0 finds the segment of the chunk's first item by
// binary search and every lane carries its segment index forward, so a warp
// searches once per chunk and each lane walks past every segment boundary of
// the chunk once.
constexpr int kWalkItems = 4;

// Local edge ids -> global ids: edge j of graph g (eoff[g] <= j < eoff[g+1])
// gets voff[g] added to both endpoints; local ids >= n_g set kErrBadVertex
// and become a self-loop on the graph's first vertex.
__global__ void k_batch_globalize(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                                  const uint64_t* __restrict__ eoff,
                                  const uint32_t* __restrict__ voff, uint32_t k, uint64_t m,
                                  uint64_t chunk, uint32_t* __restrict__ gsrc,
                                  uint32_t* __restrict__ gdst, unsigned* err) {
  const uint64_t c0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * chunk;
  if (c0 >= m) return;  // whole warps leave together
  const uint64_t c1 = c0 + chunk < m ? c0 + chunk : m;
  const unsigned lane = lane_id();
  uint32_t g = lane == 0 ? segment_of(eoff, k, c0) : 0u;
  g = __shfl_sync(kFull, g, 0);
  for (uint64_t j0 = c0 + lane; j0 < c1; j0 += 32 * kWalkItems) {
    uint32_t u[kWalkItems], v[kWalkItems];
#pragma unroll
    for (int q = 0; q < kWalkItems; ++q) {
      const uint64_t j = j0 + 32ull * q;
      u[q] = j < c1 ? src[j] : 0u;
      v[q] = j < c1 ? dst[j] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kWalkItems; ++q) {
      const uint64_t j = j0 + 32ull * q;
      if (j >= c1) break;
      while (g + 1 < k && __ldg(eoff + g + 1) <= j) ++g;
      const uint32_t base = __ldg(voff + g), ng = __ldg(voff + g + 1) - base;
      uint32_t a = u[q], b = v[q];
      if (a >= ng || b >= ng) {
        atomicOr(err, kErrBadVertex);
        a = b = 0;
      }
      gsrc[j] = base + a;
      gdst[j] = base + b;
    }
  }
}

// gid[v] = graph of vertex v for v < voff[k]: one warp per graph, so that a
// level whose graphs are mostly empty costs one check per graph.
__global__ void k_batch_gid(const uint32_t* __restrict__ voff, uint32_t k,
                            uint32_t* __restrict__ gid) {
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < k; g += nw) {
    const uint32_t a = __ldg(voff + g), b = __ldg(voff + g + 1);
    for (uint32_t v = a + lane_id(); v < b; v += 32) gid[v] = g;
  }
}

// Offsets of the next level: graph g's surviving nodes are the new ids of its
// range, so voff_next[g] = id(voff[g]) (g <= k; voff[k] = n has the total).
__global__ void k_batch_next_offsets(const uint32_t* __restrict__ voff,
                                     const uint64_t* __restrict__ rank, uint32_t k,
                                     uint32_t* __restrict__ voff_next) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= k; g += gridDim.x * blockDim.x) {
    uint32_t id;
    keep_rank(rank, voff[g], &id);
    voff_next[g] = id;
  }
}

// mcnt[g] += number of packed edges (a << 32 | b) whose endpoint a lies in
// graph g (gid: graph of every vertex of the level).  With `local` (k words
// of dynamic shared memory) a block first counts in shared memory and then
// adds its nonzero counts, so the global atomics no longer pile up on the
// few lines that hold the counters.
__global__ void k_batch_count_edges(const uint64_t* __restrict__ e, uint64_t m,
                                    const uint32_t* __restrict__ gid, uint32_t k, int local,
                                    uint32_t* __restrict__ mcnt) {
  extern __shared__ uint32_t s_cnt[];
  if (local) {
    for (uint32_t g = threadIdx.x; g < k; g += blockDim.x) s_cnt[g] = 0;
    __syncthreads();
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const uint32_t g = __ldg(gid + (uint32_t)(e[j] >> 32));
    atomicAdd(local ? &s_cnt[g] : &mcnt[g], 1u);
  }
  if (local) {
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < k; g += blockDim.x)
      if (s_cnt[g]) atomicAdd(&mcnt[g], s_cnt[g]);
  }
}

// labels[v] -= voff[graph of v]: global labels to per-graph local labels
// (vertex chunks per warp as in k_batch_globalize).
__global__ void k_batch_localize(uint32_t* __restrict__ labels, uint32_t n,
                                 const uint32_t* __restrict__ voff, uint32_t k, uint64_t chunk) {
  const uint64_t c0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * chunk;
  if (c0 >= n) return;  // whole warps leave together
  const uint64_t c1 = c0 + chunk < n ? c0 + chunk : n;
  uint32_t g = lane_id() == 0 ? segment_of(voff, k, c0) : 0u;
  g = __shfl_sync(kFull, g, 0);
  for (uint64_t v = c0 + lane_id(); v < c1; v += 32) {
    while (g + 1 < k && __ldg(voff + g + 1) <= v) ++g;
    labels[v] -= __ldg(voff + g);
  }
}

// ------------------------------------------------------- pointer jumping

// Root bitmap: bit v of isroot is set when v's stored pointer is v itself.
// Roots stay roots while the chase compresses the other pointers, so the
// bitmap stays exact during k_jump; at one bit per vertex (8 MB at n = 2^26)
// it sits in L2, where the 8-byte pointers of a large phase do not.
__global__ void __launch_bounds__(kThreads) k_root_bits(const unsigned long long* __restrict__ minkey,
                                                        uint32_t n, uint32_t* __restrict__ isroot) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // whole warps step together over 32 consecutive vertices (one bitmap word)
  for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); v0 < n;
       v0 += stride) {
    const uint64_t v = v0 + lane_id();
    const bool r = v < n && (uint32_t)minkey[v] == (uint32_t)v;
    const unsigned bits = __ballot_sync(kFull, r);
    if (lane_id() == 0) isroot[v0 >> 5] = bits;
  }
}

// kBits: consult the root bitmap (k_root_bits) before reading a pointer.
template <bool kBits>
__global__ void __launch_bounds__(kThreads) k_jump(unsigned long long* minkey,
                                                   uint32_t* __restrict__ root,
                                                   uint32_t* mo, uint32_t n,
                                                   const uint32_t* __restrict__ isroot,
                                                   unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint32_t p0 = (uint32_t)minkey[v];
    if (!index_ok(err, kKJump, p0, n)) {
      root[v] = (uint32_t)v;
      continue;
    }
    uint32_t p = p0;
    if (p != (uint32_t)v) {
      // every stored pointer leads to an ancestor, so chasing ends at the
      // root (the only vertex whose stored pointer is itself) within n steps;
      // with kBits the root bitmap answers "is p a root" from L2, so a vertex
      // whose parent is a root reads no other vertex's pointer; the checks
      // only guard against corrupted data
      uint32_t steps = 0;
      while (!kBits || !((__ldg(isroot + (p >> 5)) >> (p & 31u)) & 1u)) {
        const uint32_t q = (uint32_t)minkey[p];
        if (q == p) break;
        if (!index_ok(err, kKJump, q, n) || !index_ok(err, kKJump, ++steps, (uint64_t)n + 1))
          break;
        p = q;
      }
      // compress: later chases through v go straight to the root
      if (p != p0) minkey[v] = p;
      min_if_lower(&mo[p], mo[v]);
    }
    root[v] = p;
  }
}

// ------------------------------------------------------- phase variants

// Edge visitor over uint32 pairs (phase 0: ids validated, bad ids set
// kErrBadVertex and are skipped) or packed uint64 edges (ids checked).
template <class Op>
__global__ void __launch_bounds__(kThreads) k_for_edges(const uint32_t* __restrict__ src,
                                                        const uint32_t* __restrict__ dst,
                                                        const uint64_t* __restrict__ packed,
                                                        uint64_t m, uint32_t n, Op op,
                                                        unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    uint32_t u, v;
    if (packed != nullptr) {
      const uint64_t x = __ldcs(packed + j);
      u = (uint32_t)(x >> 32);
      v = (uint32_t)x;
      if (!index_ok(err, Op::kKernel, max(u, v), n)) continue;
    } else {
      u = __ldcs(src + j);
      v = __ldcs(dst + j);
      if (u >= n || v >= n) {
        atomicOr(err, kErrBadVertex);
        continue;
      }
    }
    op(u, v);
  }
}

// Second hop of the two-hop label (Section 3, LocalContraction):
// mk2[v] = min over u in N(v) of mk1[u], starting from mk2 = mk1.  Only the
// endpoint with the larger mk1 can improve (mk2 <= mk1), so one atomic.
__device__ __forceinline__ void two_hop_apply(uint32_t u, uint32_t v, unsigned long long a,
                                              unsigned long long b, unsigned long long* mk2) {
  if (a < b) min_if_lower(&mk2[v], a);
  else if (b < a) min_if_lower(&mk2[u], b);
}

// Edges as uint32 arrays (phase 0; `vec` = 16-byte aligned; ids >= n were
// reported by edge_min and are skipped) or packed (a << 32 | b).  mk1[u] is
// the key of f(u), so the kernel gathers the 4-byte f (fpar, half the bytes
// of mk1, so more of it stays in L2) and recomputes the keys.  Four edges per
// iteration, their eight gathers issued before any update.
template <class K>
__global__ void __launch_bounds__(kThreads) k_two_hop(const uint32_t* __restrict__ src,
                                                      const uint32_t* __restrict__ dst,
                                                      const uint64_t* __restrict__ packed,
                                                      uint64_t m, uint32_t n, int vec, K keys,
                                                      const uint32_t* __restrict__ fpar,
                                                      unsigned long long* mk2, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nq = (packed != nullptr || vec) ? m / 4 : 0;
  for (uint64_t q = gt; q < nq; q += stride) {
    uint32_t u[4], v[4];
    if (packed != nullptr) {
      const ulonglong2* e2 = reinterpret_cast<const ulonglong2*>(packed);
      const ulonglong2 p0 = __ldcs(e2 + 2 * q), p1 = __ldcs(e2 + 2 * q + 1);
      const uint64_t x[4] = {p0.x, p0.y, p1.x, p1.y};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        u[i] = (uint32_t)(x[i] >> 32);
        v[i] = (uint32_t)x[i];
      }
    } else {
      const uint4 s = __ldcs(reinterpret_cast<const uint4*>(src) + q);
      const uint4 d = __ldcs(reinterpret_cast<const uint4*>(dst) + q);
      u[0] = s.x; u[1] = s.y; u[2] = s.z; u[3] = s.w;
      v[0] = d.x; v[1] = d.y; v[2] = d.z; v[3] = d.w;
    }
    bool ok[4];
    uint32_t fu[4], fv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ok[i] = packed != nullptr ? index_ok(err, kKTwoHop, max(u[i], v[i]), n)
                                : (u[i] < n && v[i] < n);
      fu[i] = ok[i] ? __ldg(fpar + u[i]) : 0u;
      fv[i] = ok[i] ? __ldg(fpar + v[i]) : 0u;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!ok[i] || fu[i] == fv[i]) continue;
      uint64_t a, b;
      keys.pair(fu[i], fv[i], a, b);  // f(u), f(v) lie in u's graph
      two_hop_apply(u[i], v[i], a, b, mk2);
    }
  }
  for (uint64_t j = nq * 4 + gt; j < m; j += stride) {
    uint32_t u, v;
    if (packed != nullptr) {
      const uint64_t x = __ldcs(packed + j);
      u = (uint32_t)(x >> 32);
      v = (uint32_t)x;
      if (!index_ok(err, kKTwoHop, max(u, v), n)) continue;
    } else {
      u = __ldcs(src + j);
      v = __ldcs(dst + j);
      if (u >= n || v >= n) continue;
    }
    const uint32_t fu = __ldg(fpar + u), fv = __ldg(fpar + v);
    if (fu == fv) continue;
    uint64_t a, b;
    keys.pair(fu, fv, a, b);
    two_hop_apply(u, v, a, b, mk2);
  }
}

// Lock-free union of the endpoints' sets: the larger of the two roots is
// hooked under the smaller with a compare-and-swap (retried when another
// thread hooked it first).  parent[x] <= x always holds, so every find walks
// strictly decreasing ids, and a set's root is its smallest id.  Reads go
// through L2 (__ldcg) so that a retry sees the hooks of other SMs; a stale
// value is still an ancestor, and only the compare-and-swap decides.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t x, unsigned* err) {
  for (;;) {
    const uint32_t p = __ldcg(parent + x);
    if (p == x) return x;
    if (!index_ok(err, kKUnionFind, p, x)) return x;  // parent ids only decrease
    const uint32_t gp = __ldcg(parent + p);
    if (gp < p) parent[x] = gp;  // path halving: gp is an ancestor of x
    x = p;
  }
}

struct UnionOp {
  static constexpr int kKernel = kKUnionFind;
  uint32_t* parent;
  unsigned* err;
  uint32_t n;
  __device__ __forceinline__ void operator()(uint32_t u, uint32_t v) const {
    // each failed hook means that the larger root got a parent, so the sum of
    // the two roots found next is smaller: fewer than 2n retries
    for (uint64_t tries = 0;; ++tries) {
      const uint32_t a = uf_find(parent, u, err), b = uf_find(parent, v, err);
      if (a == b) return;
      const uint32_t hi = max(a, b), lo = min(a, b);
      if (atomicCAS(&parent[hi], hi, lo) == hi) return;
      if (!index_ok(err, kKUnionFind, tries, 2ull * n + 2)) return;
    }
  }
};

// mk2 = mk1, fpar = the low halves of mk1 (the parents f).
__global__ void k_two_hop_init(unsigned long long* __restrict__ mk2,
                               const unsigned long long* __restrict__ mk1,
                               uint32_t* __restrict__ fpar, uint32_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const unsigned long long k = mk1[v];
    mk2[v] = k;
    fpar[v] = (uint32_t)k;
  }
}

// Two-hop names: root[v] = the label vertex low32(mk2[v]); nmo[name] = min of
// the members' mo (a label vertex need not belong to its own group, so the
// node minima live in their own array).
__global__ void k_two_hop_names(const unsigned long long* __restrict__ mk2, uint32_t* root,
                                const uint32_t* __restrict__ mo, uint32_t* nmo, uint32_t n,
                                unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t name = (uint32_t)mk2[v];
    if (!index_ok(err, kKTwoHop, name, n)) name = (uint32_t)v;
    root[v] = name;
    min_if_lower(&nmo[name], mo[v]);
  }
}

// TreeContraction names: follow f (f(x) = low32(minkey[x]), or x itself when
// x has no other neighbour) to the terminal 2-cycle {p, f(p)} (Lemma
// lem:cycle) and name the weakly connected component by the lower-key vertex
// of that pair (Lemma lem:wccs).  The name is a member of its own group, so
// node minima are aggregated in place.
template <class K>
__global__ void __launch_bounds__(kThreads) k_tree_names(const unsigned long long* __restrict__ minkey,
                                                         uint32_t* root, uint32_t* mo, uint32_t n,
                                                         K keys, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  auto f = [&](uint32_t x) -> uint32_t {
    const unsigned long long k = minkey[x];
    return k == ~0ull ? x : (uint32_t)k;
  };
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t p = f((uint32_t)v);
    bool ok = index_ok(err, kKTreeNames, p, n);
    for (uint32_t steps = 0; ok; ++steps) {
      const uint32_t q = f(p);
      if (!index_ok(err, kKTreeNames, q, n) || !index_ok(err, kKTreeNames, steps, (uint64_t)n + 2)) {
        ok = false;
        break;
      }
      if (f(q) == p) break;  // p lies on the 2-cycle {p, q} (or q == p: no neighbour)
      p = q;
    }
    uint32_t name = (uint32_t)v;
    if (ok) {
      const uint32_t q = f(p);
      name = (q == p || keys.key(p) < keys.key(q)) ? p : q;
    }
    root[v] = name;
    if (name != (uint32_t)v) min_if_lower(&mo[name], mo[v]);
  }
}

__global__ void k_uf_init(uint32_t* parent, uint32_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    parent[v] = (uint32_t)v;
}

// Root of v once all unions are done (parents only decrease along a path).
__device__ __forceinline__ uint32_t uf_root(const uint32_t* parent, uint32_t v, unsigned* err) {
  uint32_t r = v;
  for (;;) {
    const uint32_t p = parent[r];
    if (p == r) return r;
    if (!index_ok(err, kKUnionFind, p, r)) return v;
    r = p;
  }
}

// Node minima of the union-find components, aggregated at the roots.
__global__ void k_uf_names(const uint32_t* parent, uint32_t* mo, uint32_t n, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint32_t r = uf_root(parent, (uint32_t)v, err);
    if (r != (uint32_t)v) min_if_lower(&mo[r], mo[v]);
  }
}

// root[v] = the smallest id of v's component.
__global__ void k_uf_flatten(const uint32_t* parent, uint32_t* root, uint32_t n, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    root[v] = uf_root(parent, (uint32_t)v, err);
}

// ----------------------------------------------------------- relabel

constexpr int kRelItems = 16;
static_assert(kThreads * kRelItems == kRelabelTileEdges, "relabel tile size");

__device__ __forceinline__ void relabel_one(uint32_t u, uint32_t v, bool valid, uint32_t n,
                                            const uint32_t* __restrict__ root, int bits,
                                            uint64_t& key, bool& keep) {
  keep = false;
  if (!valid || u >= n || v >= n) return;
  uint32_t a = __ldg(root + u), b = __ldg(root + v);
  if (a == b) return;
  uint32_t lo = min(a, b), hi = max(a, b);
  key = ((uint64_t)lo << bits) | hi;
  keep = true;
}

constexpr int kRelCache = 4096;  // per-block direct-mapped cache of emitted keys

// Each block handles tiles of kThreads * kRelItems edges.  Every non-loop
// edge is counted in *mprime; its key is written only if neither the block's
// cache nor the optional device-wide cache (gcache, gmask + 1 slots, both
// direct-mapped) holds it.  A key enters the device-wide cache only from the
// thread that then writes it, and the block cache only from a thread that
// writes it or that found it in the device-wide cache, so a key is dropped
// only when a copy of it is written: the written keys contain every distinct
// key.  Heavily repeated keys (pairs of large trees) are thus written a few
// times instead of once per edge, which shrinks the deduplication.  The
// written keys are compacted with a block scan and appended after one
// atomicAdd per tile.
// Half-resolved endpoint: the root id with this bit set (ids < 2^31 only).
constexpr uint32_t kResolved = 0x80000000u;

// First half of a two-pass relabel of the input edges: every endpoint below
// `split` is replaced by its root and flagged kResolved, the others are kept;
// out[j] = (a << 32 | b).  Each pass gathers from one half of `root`, which
// fits in L2.  Ids >= n become a flagged self-loop (dropped later).
__global__ void __launch_bounds__(kThreads) k_relabel_first_half(
    const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m, uint32_t n,
    uint32_t split, const uint32_t* __restrict__ root, uint64_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    uint32_t u = __ldcs(src + j), v = __ldcs(dst + j);
    uint32_t a, b;
    if (u >= n || v >= n) {
      a = b = kResolved;
    } else {
      a = u < split ? (__ldg(root + u) | kResolved) : u;
      b = v < split ? (__ldg(root + v) | kResolved) : v;
    }
    __stcs(out + j, ((uint64_t)a << 32) | b);
  }
}

// Middle pass of a relabel in more than two parts: endpoints of the
// half-resolved edges in tmp that are still unresolved and lie in [lo, hi)
// are replaced by their roots and flagged, in place.
__global__ void __launch_bounds__(kThreads) k_relabel_mid(uint64_t* __restrict__ tmp, uint64_t m,
                                                          uint32_t n, uint32_t lo, uint32_t hi,
                                                          const uint32_t* __restrict__ root,
                                                          unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const uint64_t x = tmp[j];
    uint32_t a = (uint32_t)(x >> 32), b = (uint32_t)x;
    bool changed = false;
    if (!(a & kResolved) && a - lo < hi - lo && index_ok(err, kKRelabelSplit, a, n)) {
      a = __ldg(root + a) | kResolved;
      changed = true;
    }
    if (!(b & kResolved) && b - lo < hi - lo && index_ok(err, kKRelabelSplit, b, n)) {
      b = __ldg(root + b) | kResolved;
      changed = true;
    }
    if (changed) tmp[j] = ((uint64_t)a << 32) | b;
  }
}

// kMode 0: uint32 src/dst; 1: packed (a << 32 | b); 2: packed half-resolved
// (see k_relabel_first_half).
template <int kMode>
__global__ void __launch_bounds__(kThreads) k_relabel(
    const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
    const uint64_t* __restrict__ packed, uint64_t m, uint32_t n, const uint32_t* __restrict__ root,
    int bits, uint64_t* __restrict__ keys_out, unsigned long long* mprime,
    unsigned long long* emitted, int mix, PassPlan plan, uint32_t* __restrict__ ghist,
    unsigned* mprime_err, unsigned long long* gcache, uint32_t gmask, int admit,
    unsigned* ticket, const uint64_t* __restrict__ tiles, const unsigned long long* d_ntiles) {
  __shared__ uint64_t cache[kRelCache];
  __shared__ uint32_t hist[3][kRadixMax];
  __shared__ uint32_t ws[kThreads / 32];
  __shared__ uint32_t wk[kThreads / 32];
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_t;
  const uint64_t tile_edges = (uint64_t)kThreads * kRelItems;
  // with a tile list (chunk-local grouping, packed edges only): tile t covers
  // edges [tiles[2t], tiles[2t+1]), at most tile_edges of them
  const uint64_t ntiles =
      (kMode == 1 && tiles != nullptr) ? *d_ntiles : (m + tile_edges - 1) / tile_edges;
  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  for (int i = tid; i < kRelCache; i += kThreads) cache[i] = ~0ull;
  for (int i = tid; i < 3 * kRadixMax; i += kThreads) (&hist[0][0])[i] = 0;
  __syncthreads();
  for (;;) {
    // tiles claimed in order by ticket, so the tiles in flight stay close in
    // the edge order (on grouped edges: one pair of vertex blocks, whose
    // roots stay in L2); the previous tile's closing barrier orders this
    // write after every thread's read of s_t
    if (tid == 0) s_t = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint64_t t = s_t;
    if (t >= ntiles) break;
    uint64_t tb = t * tile_edges, te = m;
    if (kMode == 1 && tiles != nullptr) {
      tb = tiles[2 * t];
      te = tiles[2 * t + 1];
      if (!index_ok(mprime_err, kKRelabelPacked, te, m + 1) ||
          !index_ok(mprime_err, kKRelabelPacked, te - tb, tile_edges + 1))
        te = tb;  // corrupted entry: the tile does nothing
    }
    // thread item i handles edge base + w*32*kRelItems + i*32 + lane (coalesced)
    const uint64_t base = tb + (uint64_t)w * 32 * kRelItems;
    uint64_t key[kRelItems];
    uint32_t keepmask = 0, emitmask = 0;
#pragma unroll
    for (int i = 0; i < kRelItems; ++i) {
      uint64_t j = base + (uint64_t)i * 32 + lane;
      bool valid = j < te;
      uint32_t u = 0, v = 0;
      if (valid) {
        if (kMode != 0) {
          uint64_t x = __ldcs(packed + j);
          u = (uint32_t)(x >> 32);
          v = (uint32_t)x;
        } else {
          u = __ldcs(src + j);
          v = __ldcs(dst + j);
        }
      }
      bool keep;
      key[i] = 0;
      if (kMode == 1 && valid &&
          !index_ok(mprime_err, kKRelabelPacked, max(u, v), n))
        valid = false;
      if (kMode == 2) {
        if (valid && (!index_ok(mprime_err, kKRelabelSoa, (u & kResolved) ? 0u : u, n) ||
                      !index_ok(mprime_err, kKRelabelSoa, (v & kResolved) ? 0u : v, n)))
          valid = false;
        uint32_t a = !valid ? 0u : (u & kResolved) ? (u & ~kResolved) : __ldg(root + u);
        uint32_t b = !valid ? 0u : (v & kResolved) ? (v & ~kResolved) : __ldg(root + v);
        keep = valid && a != b;
        if (keep) key[i] = ((uint64_t)min(a, b) << bits) | max(a, b);
      } else {
        relabel_one(u, v, valid, n, root, bits, key[i], keep);
      }
      keepmask |= (keep ? 1u : 0u) << i;
    }
#pragma unroll
    for (int i = 0; i < kRelItems; ++i) {
      if (keepmask & (1u << i)) {
        uint64_t y = key_mix(key[i]);
        uint32_t slot = (uint32_t)y & (kRelCache - 1);
        if (mix) key[i] = y;
        if (cache[slot] != key[i]) {
          cache[slot] = key[i];
          bool emit = true;
          if (gcache != nullptr) {
            // device-wide cache (slot from other bits than the block's); a
            // missing key is admitted for one in 2^admit of its occurrences
            // (chosen by the edge's position), so that keys seen once rarely
            // evict repeated ones
            unsigned long long* g = gcache + ((uint32_t)(y >> 20) & gmask);
            if (__ldcg(g) == key[i]) {
              emit = false;
            } else {
              const uint64_t j = base + (uint64_t)i * 32 + lane;
              if (admit == 0 || ((j * kGamma) >> (64 - admit)) == 0)
                __stcg(g, (unsigned long long)key[i]);
            }
          }
          if (emit) {
            emitmask |= 1u << i;
#pragma unroll
            for (int p = 0; p < 3; ++p)
              if (p < plan.passes) atomicAdd(&hist[p][plan.digit(p, key[i])], 1u);
          }
        }
      }
    }
    // warp totals, then one block scan over them; a warp writes the emitted
    // keys of each item position as one contiguous run (coalesced stores)
    uint32_t wtot = 0;
    uint32_t kept = __popc(keepmask);
#pragma unroll
    for (int i = 0; i < kRelItems; ++i) wtot += __popc(__ballot_sync(kFull, (emitmask >> i) & 1u));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) kept += __shfl_xor_sync(kFull, kept, o);
    if (lane == 0) {
      ws[w] = wtot;
      wk[w] = kept;
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t run = 0, kall = 0;
      for (int k = 0; k < kThreads / 32; ++k) {
        uint32_t c = ws[k];
        ws[k] = run;
        run += c;
        kall += wk[k];
      }
      if (kall) atomicAdd(mprime, (unsigned long long)kall);
      s_base = run ? atomicAdd(emitted, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    uint64_t pos = s_base + ws[w];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kRelItems; ++i) {
      const unsigned b = __ballot_sync(kFull, (emitmask >> i) & 1u);
      if ((emitmask >> i) & 1u) __stcs(keys_out + pos + __popc(b & lt), key[i]);
      pos += __popc(b);
    }
    __syncthreads();
  }
  for (int i = tid; i < plan.passes * kRadixMax; i += kThreads) {
    uint32_t c = (&hist[0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// ------------------------------------------------------ label composition

__global__ void __launch_bounds__(kThreads) k_propagate(const uint32_t* root,
                                                        const uint64_t* __restrict__ rank,
                                                        const uint32_t* __restrict__ mo,
                                                        const uint32_t* __restrict__ labels_up,
                                                        uint32_t* labels_out, uint32_t n,
                                                        uint32_t n_up, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t r = root[v];
    if (!index_ok(err, kKPropagate, r, n)) {
      labels_out[v] = (uint32_t)v;
      continue;
    }
    uint32_t s0;
    const bool kept = keep_rank(rank, r, &s0);
    if (kept && !index_ok(err, kKPropagate, s0, n_up)) {
      labels_out[v] = (uint32_t)v;
      continue;
    }
    labels_out[v] = kept ? labels_up[s0] : mo[r];
  }
}

__global__ void k_stamp(Counters* ctr, unsigned long long tag) { ctr->tag = tag; }

__global__ void k_identity(uint32_t* labels, uint32_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    labels[v] = (uint32_t)v;
}

}  // namespace

void init_keys(unsigned long long* minkey, uint32_t* mo, uint32_t n, uint64_t rk,
               const BatchView* batch, const Launch& L) {
  if (n == 0) return;
  KScope ks(L, kKInitKeys);
  if (batch)
    k_init_keys<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(
        minkey, mo, n, BatchKeys{batch->gs, batch->voff, batch->k, batch->gid});
  else
    k_init_keys<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(minkey, mo, n, GraphKeys{rk});
}

template <bool kOpen, class K>
static void edge_min_impl(const uint32_t* src, const uint32_t* dst, const uint64_t* packed,
                          uint64_t m, uint32_t n, K keys, unsigned long long* minkey,
                          unsigned* err, uint64_t window_bytes, const Launch& L) {
  if (packed != nullptr) {
    KScope ks(L, kOpen ? kKOpenMin : kKEdgeMinPacked);
    k_edge_min_packed<kOpen><<<grid_for(m / 2 + 1, kThreads, L), kThreads, 0, L.stream>>>(
        packed, m, keys, minkey, n, err);
  } else {
    int vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    // vertex windows whose minkey slices fit the L2 budget; one pass each
    uint64_t wv = std::max<uint64_t>(1, window_bytes / 8);
    uint32_t passes = (uint32_t)std::max<uint64_t>(1, (n + wv - 1) / wv);
    uint64_t span = ((uint64_t)n + passes - 1) / passes;
    for (uint32_t p = 0; p < passes; ++p) {
      uint64_t lo = (uint64_t)p * span;
      uint64_t sp = std::min<uint64_t>(span, n - lo);
      KScope ks(L, kOpen ? kKOpenMin : kKEdgeMinSoa);
      k_edge_min_soa<kOpen><<<grid_for((m + 3) / 4, kThreads, L), kThreads, 0, L.stream>>>(
          src, dst, m, n, keys, minkey, err, vec, (uint32_t)lo, (uint32_t)sp, p == 0);
    }
  }
}

void edge_min(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
              uint32_t n, uint64_t rk, unsigned long long* minkey, unsigned* err,
              uint64_t window_bytes, const BatchView* batch, const Launch& L, bool open) {
  if (m == 0) return;
  if (batch) {
    const BatchKeys k{batch->gs, batch->voff, batch->k, batch->gid};
    if (open) edge_min_impl<true>(src, dst, packed, m, n, k, minkey, err, window_bytes, L);
    else edge_min_impl<false>(src, dst, packed, m, n, k, minkey, err, window_bytes, L);
  } else {
    const GraphKeys k{rk};
    if (open) edge_min_impl<true>(src, dst, packed, m, n, k, minkey, err, window_bytes, L);
    else edge_min_impl<false>(src, dst, packed, m, n, k, minkey, err, window_bytes, L);
  }
}

// Items per warp of the chunked walks (a multiple of 32), for `grid` blocks.
static uint64_t walk_chunk(uint64_t items, int grid) {
  const uint64_t warps = (uint64_t)grid * (kThreads / 32);
  const uint64_t per = (items + warps - 1) / warps;
  return (per + 31) / 32 * 32;
}

// Largest k whose per-graph edge counts a block keeps in shared memory.
constexpr uint32_t kCountLocalMax = 8192;

void batch_phase_seeds(const uint64_t* seeds, uint32_t k, uint32_t i, const uint32_t* voff,
                       uint64_t* gs, const Launch& L) {
  KScope ks(L, kKBatch);
  k_batch_phase_seeds<<<grid_for(k, kThreads, L), kThreads, 0, L.stream>>>(seeds, k, i, voff, gs);
}

void batch_globalize(const uint32_t* src, const uint32_t* dst, const uint64_t* eoff,
                     const uint32_t* voff, uint32_t k, uint64_t m, uint32_t* gsrc, uint32_t* gdst,
                     unsigned* err, const Launch& L) {
  if (m == 0) return;
  const int grid = grid_for(m, kThreads, L);
  const uint64_t chunk = walk_chunk(m, grid);
  KScope ks(L, kKBatch);
  k_batch_globalize<<<grid, kThreads, 0, L.stream>>>(src, dst, eoff, voff, k, m, chunk, gsrc,
                                                     gdst, err);
}

void batch_graph_ids(const uint32_t* voff, uint32_t k, uint32_t n, uint32_t* gid,
                     const Launch& L) {
  if (n == 0) return;
  KScope ks(L, kKBatch);
  k_batch_gid<<<grid_for(32ull * k, kThreads, L), kThreads, 0, L.stream>>>(voff, k, gid);
}

void batch_next_level(const uint32_t* voff, const uint64_t* rank, uint32_t k, uint32_t* voff_next,
                      const uint64_t* e, uint64_t m, uint32_t* mcnt, uint32_t n_next,
                      uint32_t* gid, const Launch& L) {
  {
    KScope ks(L, kKBatch);
    k_batch_next_offsets<<<grid_for(k + 1, kThreads, L), kThreads, 0, L.stream>>>(voff, rank, k,
                                                                                  voff_next);
  }
  batch_graph_ids(voff_next, k, n_next, gid, L);
  cudaMemsetAsync(mcnt, 0, sizeof(uint32_t) * k, L.stream);
  if (m) {
    KScope ks(L, kKBatch);
    const int local = k <= kCountLocalMax;
    // fewer blocks when counting locally: each block adds up to k counts
    const int grid = grid_for(m, kThreads, L, local ? 4 : 8);
    k_batch_count_edges<<<grid, kThreads, local ? 4 * k : 0, L.stream>>>(
        e, m, gid, k, local, mcnt);
  }
}

void batch_localize(uint32_t* labels, uint32_t n, const uint32_t* voff, uint32_t k,
                    const Launch& L) {
  if (n == 0) return;
  const int grid = grid_for(n, kThreads, L);
  const uint64_t chunk = walk_chunk(n, grid);
  KScope ks(L, kKBatch);
  k_batch_localize<<<grid, kThreads, 0, L.stream>>>(labels, n, voff, k, chunk);
}

void jump(unsigned long long* minkey, uint32_t* root, uint32_t* mo, uint32_t n, uint64_t m,
          uint32_t* isroot, uint32_t bits_min_vertices, unsigned* err, const Launch& L) {
  if (n == 0) return;
  KScope ks(L, kKJump);
  // The bitmap pays when the pointers do not fit L2 and the forest is deep
  // and scattered, as on sparse graphs (grids, meshes: average degree below
  // 4); on skewed dense graphs most parents are a few hubs, whose pointers
  // L2 already holds, and the extra pass and bitmap reads only cost.
  if (isroot != nullptr && n >= bits_min_vertices && m < 4ull * n) {
    k_root_bits<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(minkey, n, isroot);
    k_jump<true><<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(minkey, root, mo, n,
                                                                      isroot, err);
  } else {
    k_jump<false><<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(minkey, root, mo, n,
                                                                       nullptr, err);
  }
}

void relabel(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
             uint32_t n, const uint32_t* root, int bits, uint64_t* keys_out,
             unsigned long long* mprime, unsigned long long* emitted, bool mix,
             const PassPlan* plan, uint32_t* ghist, uint64_t* tmp, uint64_t window_bytes,
             unsigned long long* gcache, uint32_t gslots, int admit, unsigned* ticket,
             unsigned* err, const Launch& L, const uint64_t* tiles,
             const unsigned long long* d_ntiles) {
  const uint32_t gmask = gslots ? gslots - 1 : 0;
  if (gslots == 0) gcache = nullptr;
  PassPlan pl{};
  if (plan != nullptr) pl = *plan;  // passes == 0: no histogram
  if (m == 0) return;
  int grid = grid_for(m, kThreads * kRelItems, L, 4);
  cudaMemsetAsync(ticket, 0, sizeof(unsigned), L.stream);
  if (packed != nullptr) {
    KScope ks(L, kKRelabelPacked);
    k_relabel<1><<<grid, kThreads, 0, L.stream>>>(nullptr, nullptr, packed, m, n, root, bits,
                                                  keys_out, mprime, emitted, mix, pl, ghist,
                                                  err, gcache, gmask, admit, ticket, tiles,
                                                  d_ntiles);
  } else if (tmp != nullptr && n < kResolved && (uint64_t)n * 4 > window_bytes) {
    // one pass per L2-sized part of root (see k_relabel_first_half)
    const uint64_t parts = std::min<uint64_t>(8, ((uint64_t)n * 4 + window_bytes - 1) /
                                                     std::max<uint64_t>(window_bytes, 1));
    auto cut = [&](uint64_t k) { return (uint32_t)((uint64_t)n * k / parts); };
    {
      KScope ks(L, kKRelabelSplit);
      k_relabel_first_half<<<grid_for(m, kThreads, L), kThreads, 0, L.stream>>>(src, dst, m, n,
                                                                               cut(1), root, tmp);
    }
    for (uint64_t k = 1; k + 1 < parts; ++k) {
      KScope ks(L, kKRelabelSplit);
      k_relabel_mid<<<grid_for(m, kThreads, L), kThreads, 0, L.stream>>>(tmp, m, n, cut(k),
                                                                        cut(k + 1), root, err);
    }
    KScope ks(L, kKRelabelSoa);
    k_relabel<2><<<grid, kThreads, 0, L.stream>>>(nullptr, nullptr, tmp, m, n, root, bits,
                                                  keys_out, mprime, emitted, mix, pl, ghist,
                                                  err, gcache, gmask, admit, ticket, nullptr,
                                                  nullptr);
  } else {
    KScope ks(L, kKRelabelSoa);
    k_relabel<0><<<grid, kThreads, 0, L.stream>>>(src, dst, nullptr, m, n, root, bits, keys_out,
                                                  mprime, emitted, mix, pl, ghist, err, gcache,
                                                  gmask, admit, ticket, nullptr, nullptr);
  }
}

void propagate(const uint32_t* root, const uint64_t* rank, const uint32_t* mo,
               const uint32_t* labels_up, uint32_t* labels_out, uint32_t n, uint32_t n_up,
               unsigned* err, const Launch& L) {
  if (n == 0) return;
  KScope ks(L, kKPropagate);
  k_propagate<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(root, rank, mo, labels_up,
                                                                   labels_out, n, n_up, err);
}

void stamp_counters(Counters* ctr, uint64_t tag, const Launch& L) {
  KScope ks(L, kKBatch);
  k_stamp<<<1, 1, 0, L.stream>>>(ctr, tag);
}

template <class Op>
static void for_edges(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
                      uint32_t n, Op op, unsigned* err, const Launch& L) {
  if (m == 0) return;
  KScope ks(L, Op::kKernel);
  k_for_edges<<<grid_for(m, kThreads, L), kThreads, 0, L.stream>>>(src, dst, packed, m, n, op,
                                                                   err);
}

template <class K>
static void two_hop_impl(const uint32_t* src, const uint32_t* dst, const uint64_t* packed,
                         uint64_t m, uint32_t n, K keys, const uint32_t* fpar,
                         unsigned long long* mk2, unsigned* err, const Launch& L) {
  const int vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
  KScope ks(L, kKTwoHop);
  k_two_hop<<<grid_for((m + 3) / 4, kThreads, L), kThreads, 0, L.stream>>>(
      src, dst, packed, m, n, vec, keys, fpar, mk2, err);
}

void two_hop_names(const uint32_t* src, const uint32_t* dst, const uint64_t* packed, uint64_t m,
                   uint32_t n, uint64_t rk, const BatchView* batch,
                   const unsigned long long* mk1, unsigned long long* mk2, uint32_t* fpar,
                   uint32_t* root, const uint32_t* mo, uint32_t* nmo, unsigned* err,
                   const Launch& L) {
  if (n == 0) return;
  {
    KScope ks(L, kKTwoHop);
    k_two_hop_init<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(mk2, mk1, fpar, n);
  }
  if (m) {
    if (batch)
      two_hop_impl(src, dst, packed, m, n, BatchKeys{batch->gs, batch->voff, batch->k, batch->gid}, fpar,
                   mk2, err, L);
    else
      two_hop_impl(src, dst, packed, m, n, GraphKeys{rk}, fpar, mk2, err, L);
  }
  cudaMemsetAsync(nmo, 0xFF, sizeof(uint32_t) * n, L.stream);
  KScope ks(L, kKTwoHop);
  k_two_hop_names<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(mk2, root, mo, nmo, n,
                                                                       err);
}

void tree_names(const unsigned long long* minkey, uint32_t* root, uint32_t* mo, uint32_t n,
                uint64_t rk, const BatchView* batch, unsigned* err, const Launch& L) {
  if (n == 0) return;
  KScope ks(L, kKTreeNames);
  if (batch)
    k_tree_names<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(
        minkey, root, mo, n, BatchKeys{batch->gs, batch->voff, batch->k, batch->gid}, err);
  else
    k_tree_names<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(minkey, root, mo, n,
                                                                      GraphKeys{rk}, err);
}

void union_find_names(const uint32_t* src, const uint32_t* dst, const uint64_t* packed,
                      uint64_t m, uint32_t n, uint32_t* parent, uint32_t* root, uint32_t* mo,
                      unsigned* err, const Launch& L) {
  if (n == 0) return;
  {
    KScope ks(L, kKUnionFind);
    k_uf_init<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(parent, n);
  }
  for_edges(src, dst, packed, m, n, UnionOp{parent, err, n}, err, L);
  {
    KScope ks(L, kKUnionFind);
    k_uf_names<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(parent, mo, n, err);
  }
  KScope ks(L, kKUnionFind);
  k_uf_flatten<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(parent, root, n, err);
}

void identity_labels(uint32_t* labels, uint32_t n, const Launch& L) {
  if (n == 0) return;
  KScope ks(L, kKIdentity);
  k_identity<<<grid_for(n, kThreads, L), kThreads, 0, L.stream>>>(labels, n);
}

void rank_probe(uint64_t rk, uint32_t v0, uint32_t count, uint32_t* out, const Launch& L) {
  if (count == 0) return;
  KScope ks(L, kKRankProbe);
  k_rank_probe<<<grid_for(count, kThreads, L), kThreads, 0, L.stream>>>(rk, v0, count, out);
}

}  // namespace lc
