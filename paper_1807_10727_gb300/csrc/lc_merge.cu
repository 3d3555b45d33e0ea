// MergeToLarge step (arXiv 1807.10727, Section 5): after a phase has
// contracted G_i into G' (n' nodes, packed edges), every node of G' that was
// formed from at least alpha vertices of G_i is large, with priority = the
// alpha-th largest phase-i key among those vertices; every other node that has
// a large node at distance 1 or 2 in G' joins the large node of highest
// priority.  The result is a node map t over G' (a contraction level like the
// phase's own), which the caller contracts with the usual relabel / dedup /
// compaction steps.
#include <algorithm>

#include "lc_internal.cuh"

namespace lc {
namespace {

constexpr int kThreads = 256;
constexpr int kSelThreads = 256;
constexpr int kDigits = 256;
// Large nodes with at least this many members take the first digit of their
// select from the whole grid (k_m2l_big_*), not from one block.
constexpr uint32_t kBigGroup = 1u << 15;

inline int grid_for(uint64_t work, int per_block, const Launch& L, int blocks_per_sm = 8) {
  uint64_t b = (work + per_block - 1) / per_block;
  uint64_t cap = (uint64_t)L.sms * blocks_per_sm;
  return (int)std::max<uint64_t>(1, std::min(b, cap));
}

// Node of G' that vertex v of G_i was contracted into, or n' when v's node
// was dropped (it kept no edge).
__device__ __forceinline__ uint32_t node_of(const uint32_t* root, const uint64_t* rank,
                                            uint32_t v, uint32_t n_i, uint32_t n2, unsigned* err,
                                            int kernel) {
  const uint32_t r = root[v];
  if (!index_ok(err, kernel, r, n_i)) return n2;
  uint32_t s0;
  if (!keep_rank(rank, r, &s0)) return n2;
  return index_ok(err, kernel, s0, n2) ? s0 : n2;
}

// cnt[x] = number of G_i vertices contracted into node x.
__global__ void k_m2l_count(const uint32_t* __restrict__ root, const uint64_t* __restrict__ rank,
                            uint32_t n_i, uint32_t n2, uint32_t* cnt, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_i; v += stride) {
    const uint32_t x = node_of(root, rank, (uint32_t)v, n_i, n2, err, kKMergeGroup);
    if (x < n2) atomicAdd(&cnt[x], 1u);
  }
}

// Large nodes: a segment [off[x], off[x] + cnt[x]) of the member array each
// (segments in any order) and an entry in the list of large nodes.
// ctrs[0] = member slots handed out, ctrs[1] = large nodes.
// Nodes of at least kBigGroup members are also listed in big_list (ctrs[2]
// of them, at most nbig_max).
__global__ void k_m2l_large(const uint32_t* __restrict__ cnt, uint32_t n2, uint32_t alpha,
                            uint32_t* off, uint32_t* list, unsigned* ctrs, uint32_t* big_list,
                            uint32_t nbig_max, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n2; x += stride) {
    const uint32_t c = cnt[x];
    if (c >= alpha) {
      off[x] = atomicAdd(&ctrs[0], c);
      list[atomicAdd(&ctrs[1], 1u)] = (uint32_t)x;
      if (c >= kBigGroup) {
        const uint32_t j = atomicAdd(&ctrs[2], 1u);
        if (index_ok(err, kKMergeGroup, j, nbig_max)) big_list[j] = (uint32_t)x;
      }
    }
  }
}

// Big nodes, first digit over the whole grid: hist[j][d] = members of big
// node j whose key's top byte is d.
__global__ void __launch_bounds__(kSelThreads) k_m2l_big_hist(
    const uint32_t* __restrict__ members, const uint32_t* __restrict__ cnt,
    const uint32_t* __restrict__ off, const uint32_t* __restrict__ big_list, const unsigned* ctrs,
    uint32_t nbig_max, uint64_t rk, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kDigits];
  const uint32_t nbig = min(ctrs[2], nbig_max);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t j = 0; j < nbig; ++j) {
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const uint32_t x = big_list[j], c = cnt[x], o = off[x];
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < c; k += stride)
      atomicAdd(&h[phase_key(rk, members[o + k]) >> 56], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x)
      if (h[d]) atomicAdd(&hist[(uint64_t)j * kDigits + d], h[d]);
    __syncthreads();
  }
}

// One thread per big node: the top digit of its alpha-th largest key, and the
// rank still sought among the members that share it.  pick[j] = (digit, need).
__global__ void k_m2l_big_pick(const uint32_t* __restrict__ hist, const unsigned* ctrs,
                               uint32_t nbig_max, uint32_t alpha, uint2* pick, unsigned* err) {
  const uint32_t nbig = min(ctrs[2], nbig_max);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nbig;
       j += gridDim.x * blockDim.x) {
    uint32_t above = 0, sel = kDigits;
    for (int d = kDigits - 1; d >= 0; --d) {
      const uint32_t c = hist[(uint64_t)j * kDigits + d];
      if (above + c >= alpha) {
        sel = (uint32_t)d;
        break;
      }
      above += c;
    }
    if (sel == kDigits) {  // fewer than alpha members: corrupted counts
      index_ok(err, kKMergeSelect, alpha, above + 1);
      sel = 0;
      above = 0;
    }
    pick[j] = make_uint2(sel, alpha - above);
  }
}

// The members of each big node whose top byte is the picked digit, as keys,
// to the front of its cand segment (bigcnt[j] of them).
__global__ void __launch_bounds__(kSelThreads) k_m2l_big_compact(
    const uint32_t* __restrict__ members, const uint32_t* __restrict__ cnt,
    const uint32_t* __restrict__ off, const uint32_t* __restrict__ big_list, const unsigned* ctrs,
    uint32_t nbig_max, uint64_t rk, const uint2* __restrict__ pick, unsigned long long* cand,
    uint32_t* bigcnt, unsigned* err) {
  const uint32_t nbig = min(ctrs[2], nbig_max);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t j = 0; j < nbig; ++j) {
    const uint32_t x = big_list[j], c = cnt[x], o = off[x], sel = pick[j].x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < c; k += stride) {
      const uint64_t key = phase_key(rk, members[o + k]);
      if ((key >> 56) == sel) {
        const uint32_t q = atomicAdd(&bigcnt[j], 1u);
        if (index_ok(err, kKMergeSelect, q, c)) cand[o + q] = key;
      }
    }
  }
}

// members[off[x] + j] = the j-th (in any order) G_i vertex of large node x.
__global__ void k_m2l_scatter(const uint32_t* __restrict__ root, const uint64_t* __restrict__ rank,
                              uint32_t n_i, uint32_t n2, const uint32_t* __restrict__ cnt,
                              const uint32_t* __restrict__ off, uint32_t alpha, uint32_t* fill,
                              uint32_t* members, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_i; v += stride) {
    const uint32_t x = node_of(root, rank, (uint32_t)v, n_i, n2, err, kKMergeGroup);
    if (x >= n2 || cnt[x] < alpha) continue;
    const uint32_t j = atomicAdd(&fill[x], 1u);
    const uint64_t pos = (uint64_t)off[x] + j;
    if (index_ok(err, kKMergeGroup, j, cnt[x]) && index_ok(err, kKMergeGroup, pos, n_i))
      members[pos] = (uint32_t)v;
  }
}

// Priority of every large node: the alpha-th largest phase-i key of its
// members, by a most-significant-digit-first radix select (8-bit digits) run
// by one block per node.  The first digit is taken over all members; the
// members that share it are copied (as keys) to cand, and the other seven
// digits are taken over those.  prio[x] = key + 1 (0 marks a small node).
// big_mode: only the big nodes, whose first digit, remaining rank and
// candidates the k_m2l_big_* kernels produced.
__global__ void __launch_bounds__(kSelThreads) k_m2l_select(
    const uint32_t* __restrict__ members, unsigned long long* cand,
    const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off,
    const uint32_t* __restrict__ list, const unsigned* ctrs, uint32_t alpha, uint64_t rk,
    unsigned long long* prio, unsigned* err, int big_mode, const uint32_t* __restrict__ big_list,
    uint32_t nbig_max, const uint2* __restrict__ pick, const uint32_t* __restrict__ bigcnt) {
  __shared__ uint32_t hist[kDigits];
  __shared__ uint32_t s_digit, s_need, s_ncand;
  const uint32_t count = big_mode ? min(ctrs[2], nbig_max) : ctrs[1];
  for (uint32_t j = blockIdx.x; j < count; j += gridDim.x) {
    const uint32_t x = big_mode ? big_list[j] : list[j];
    const uint32_t c = cnt[x], o = off[x];
    if (!big_mode && c >= kBigGroup) continue;  // selected in big mode
    uint64_t prefix = 0;
    uint32_t need = alpha;  // rank (1 = largest) still sought among the candidates
    uint32_t ncand = c;
    int first = 0;
    if (big_mode) {  // first digit already taken by the whole grid
      prefix = (uint64_t)pick[j].x << 56;
      need = pick[j].y;
      ncand = bigcnt[j];
      first = 1;
    }
    for (int pass = first; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      for (int d = threadIdx.x; d < kDigits; d += blockDim.x) hist[d] = 0;
      if (threadIdx.x == 0) s_ncand = 0;
      __syncthreads();
      for (uint32_t k = threadIdx.x; k < ncand; k += blockDim.x) {
        const uint64_t key = pass == 0 ? phase_key(rk, members[o + k]) : cand[o + k];
        // candidates after the first pass all share the digits above `shift`
        if (pass == 0 || (key >> (shift + 8)) == (prefix >> (shift + 8)))
          atomicAdd(&hist[(key >> shift) & 0xFF], 1u);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t above = 0, sel = kDigits;
        for (int d = kDigits - 1; d >= 0; --d) {
          if (above + hist[d] >= need) {
            sel = (uint32_t)d;
            break;
          }
          above += hist[d];
        }
        if (sel == kDigits) {  // fewer than `need` candidates: corrupted counts
          index_ok(err, kKMergeSelect, need, above + 1);
          sel = 0;
        } else {
          need -= above;
        }
        s_digit = sel;
        s_need = need;
      }
      __syncthreads();
      prefix |= (uint64_t)s_digit << shift;
      need = s_need;
      if (pass == 0) {
        // keep the members whose top digit is the selected one
        for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
          const uint64_t key = phase_key(rk, members[o + k]);
          if ((key >> 56) == s_digit) cand[o + atomicAdd(&s_ncand, 1u)] = key;
        }
        __syncthreads();
        ncand = s_ncand;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) prio[x] = prefix + 1;
    __syncthreads();
  }
}

// dst[x] = max(dst[x], src[y]) over the edges xy of G' (dst starts as src):
// only the endpoint with the smaller src value can rise, so one atomic.
__global__ void __launch_bounds__(kThreads) k_m2l_hop(const uint64_t* __restrict__ e, uint64_t m,
                                                      uint32_t n2,
                                                      const unsigned long long* __restrict__ src,
                                                      unsigned long long* dst, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const uint64_t x = __ldcs(e + j);
    const uint32_t a = (uint32_t)(x >> 32), b = (uint32_t)x;
    if (!index_ok(err, kKMergeHop, max(a, b), n2)) continue;
    const unsigned long long pa = src[a], pb = src[b];
    if (pa > pb) max_if_higher(&dst[b], pa);
    else if (pb > pa) max_if_higher(&dst[a], pb);
  }
}

__global__ void k_m2l_copy(unsigned long long* __restrict__ dst,
                           const unsigned long long* __restrict__ src, uint32_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    dst[v] = src[v];
}

// t[x] = the node that x joins: x itself when x is large or has no large
// node within distance 2, else the large node whose priority is h2[x] (a
// priority is a member's key, whose low half is that member's G_i id).  The
// target is large and never moves, so node minima are aggregated in place.
__global__ void k_m2l_target(const unsigned long long* __restrict__ prio,
                             const unsigned long long* __restrict__ h2,
                             const uint32_t* __restrict__ root, const uint64_t* __restrict__ rank,
                             uint32_t n_i, uint32_t n2, uint32_t* t, uint32_t* mo, unsigned* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n2; x += stride) {
    uint32_t y = (uint32_t)x;
    const unsigned long long h = h2[x];
    if (prio[x] == 0 && h != 0) {
      const uint32_t w = (uint32_t)(h - 1);
      if (index_ok(err, kKMergeTarget, w, n_i)) {
        const uint32_t z = node_of(root, rank, w, n_i, n2, err, kKMergeTarget);
        if (index_ok(err, kKMergeTarget, z, n2)) y = z;
      }
    }
    t[x] = y;
    if (y != (uint32_t)x) min_if_lower(&mo[y], mo[x]);
  }
}

}  // namespace

void merge_to_large_names(const uint32_t* root_i, const uint64_t* rank_i, uint32_t n_i,
                          uint64_t rk, uint32_t alpha, const uint64_t* e, uint64_t m,
                          uint32_t n2, uint32_t* t, uint32_t* mo, const MergeScratch& s,
                          unsigned* err, const Launch& L) {
  if (n2 == 0) return;
  cudaMemsetAsync(s.cnt, 0, sizeof(uint32_t) * n2, L.stream);
  cudaMemsetAsync(s.fill, 0, sizeof(uint32_t) * n2, L.stream);
  cudaMemsetAsync(s.ctrs, 0, sizeof(unsigned) * 3, L.stream);
  const uint32_t nbig_max = n_i / kBigGroup + 1;
  uint32_t* big_list = s.big;
  uint32_t* big_hist = big_list + nbig_max;
  uint32_t* bigcnt = big_hist + (uint64_t)nbig_max * kDigits;
  // 258 * nbig_max words precede it: 8-byte aligned
  uint2* pick = reinterpret_cast<uint2*>(bigcnt + nbig_max);
  cudaMemsetAsync(big_hist, 0, sizeof(uint32_t) * (uint64_t)nbig_max * (kDigits + 1), L.stream);
  cudaMemsetAsync(s.prio, 0, sizeof(unsigned long long) * n2, L.stream);
  {
    KScope ks(L, kKMergeGroup);
    k_m2l_count<<<grid_for(n_i, kThreads, L), kThreads, 0, L.stream>>>(root_i, rank_i, n_i, n2,
                                                                       s.cnt, err);
  }
  {
    KScope ks(L, kKMergeGroup);
    k_m2l_large<<<grid_for(n2, kThreads, L), kThreads, 0, L.stream>>>(
        s.cnt, n2, alpha, s.off, s.list, s.ctrs, big_list, nbig_max, err);
  }
  {
    KScope ks(L, kKMergeGroup);
    k_m2l_scatter<<<grid_for(n_i, kThreads, L), kThreads, 0, L.stream>>>(
        root_i, rank_i, n_i, n2, s.cnt, s.off, alpha, s.fill, s.members, err);
  }
  {
    KScope ks(L, kKMergeSelect);
    // at most n2 / alpha large nodes; a few blocks per multiprocessor
    const uint64_t most = std::max<uint64_t>(1, n2 / std::max<uint32_t>(alpha, 1));
    const int grid = (int)std::min<uint64_t>(most, (uint64_t)L.sms * 8);
    k_m2l_select<<<grid, kSelThreads, 0, L.stream>>>(s.members, s.cand, s.cnt, s.off, s.list,
                                                     s.ctrs, alpha, rk, s.prio, err, 0, big_list,
                                                     nbig_max, pick, bigcnt);
  }
  if ((uint64_t)n_i >= kBigGroup && alpha <= n_i) {
    // big nodes: first digit and compaction over the whole grid, then the
    // remaining digits one block per node
    const int grid = L.sms * 4;
    {
      KScope ks(L, kKMergeSelect);
      k_m2l_big_hist<<<grid, kSelThreads, 0, L.stream>>>(s.members, s.cnt, s.off, big_list,
                                                         s.ctrs, nbig_max, rk, big_hist);
    }
    {
      KScope ks(L, kKMergeSelect);
      k_m2l_big_pick<<<(nbig_max + 255) / 256, 256, 0, L.stream>>>(big_hist, s.ctrs, nbig_max,
                                                                 alpha, pick, err);
    }
    {
      KScope ks(L, kKMergeSelect);
      k_m2l_big_compact<<<grid, kSelThreads, 0, L.stream>>>(s.members, s.cnt, s.off, big_list,
                                                            s.ctrs, nbig_max, rk, pick, s.cand,
                                                            bigcnt, err);
    }
    KScope ks(L, kKMergeSelect);
    k_m2l_select<<<(int)std::min<uint32_t>(nbig_max, (uint32_t)L.sms * 8), kSelThreads, 0,
                   L.stream>>>(s.members, s.cand, s.cnt, s.off, s.list, s.ctrs, alpha, rk, s.prio,
                               err, 1, big_list, nbig_max, pick, bigcnt);
  }
  // best priority within distance 1, then within distance 2
  {
    KScope ks(L, kKMergeHop);
    k_m2l_copy<<<grid_for(n2, kThreads, L), kThreads, 0, L.stream>>>(s.h1, s.prio, n2);
  }
  if (m) {
    KScope ks(L, kKMergeHop);
    k_m2l_hop<<<grid_for(m, kThreads, L), kThreads, 0, L.stream>>>(e, m, n2, s.prio, s.h1, err);
  }
  {
    KScope ks(L, kKMergeHop);
    k_m2l_copy<<<grid_for(n2, kThreads, L), kThreads, 0, L.stream>>>(s.h2, s.h1, n2);
  }
  if (m) {
    KScope ks(L, kKMergeHop);
    k_m2l_hop<<<grid_for(m, kThreads, L), kThreads, 0, L.stream>>>(e, m, n2, s.h1, s.h2, err);
  }
  KScope ks(L, kKMergeTarget);
  k_m2l_target<<<grid_for(n2, kThreads, L), kThreads, 0, L.stream>>>(s.prio, s.h2, root_i, rank_i,
                                                                     n_i, n2, t, mo, err);
}

}  // namespace lc
