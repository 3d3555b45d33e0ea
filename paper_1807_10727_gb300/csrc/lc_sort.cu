// Onesweep LSD radix sort of 64-bit edge keys and the single-pass scans that
// compact vertices and edges (the "group by vertex / remove duplicates" shuffle
// of the O(1)-round contraction lemma, done on one GPU).
//
// Sort: Adinets and Merrill, "Onesweep: A Faster Least Significant Digit Radix
// Sort for GPUs" (2022): one pass computes the digit histograms of every pass,
// then each pass ranks a 4096-key tile in shared memory, obtains the tile's
// global digit offsets by decoupled look-back over the preceding tiles, stages
// the tile in digit order in shared memory and writes it out with coalesced
// runs.  Tiles are claimed through an atomic ticket so that every tile a block
// waits on belongs to a block that started earlier.
#include <algorithm>

#include "lc_internal.cuh"

namespace lc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = kSortThreads / 32;

// Exclusive block scan of one value per thread (kThreadsT threads, at most
// 1024).  `ws` must hold kThreadsT / 32 words; the call ends with a barrier
// so `ws` can be reused afterwards.
template <int kThreadsT = kSortThreads>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* ws,
                                                         uint32_t* total) {
  constexpr int kWarps = kThreadsT / 32;
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < (unsigned)kWarps ? ws[lane] : 0u;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, s, o);
      if (lane >= (unsigned)o) s += y;
    }
    if (lane < (unsigned)kWarps) ws[lane] = s;
  }
  __syncthreads();
  uint32_t before = w > 0 ? ws[w - 1] : 0u;
  *total = ws[kWarps - 1];
  __syncthreads();
  return before + x - v;
}

// Publishes this tile's aggregate, walks back over preceding tiles until an
// inclusive prefix is found, publishes its own inclusive prefix and returns
// the exclusive prefix.  Every wait is bounded by kSpinLimit.  After a wait
// runs out, the published prefix is only a lower bound (the offsets behind it
// come out too low, so writes stay inside the output) and kErrTimeout makes
// the host discard the phase.
__device__ __forceinline__ uint32_t look_back(uint64_t* status, uint32_t tile, uint32_t agg,
                                              uint32_t epoch, unsigned* err) {
  if (tile == 0) {
    store_status(status, pack_status(epoch, kFlagPrefix, agg));
    return 0;
  }
  store_status(status + tile, pack_status(epoch, kFlagAgg, agg));
  uint32_t excl = 0;
  uint32_t j = tile - 1;
  uint32_t spins = 0;
  for (;;) {
    uint64_t w = load_status(status + j);
    if ((uint32_t)(w >> 34) == epoch) {
      uint32_t flag = (uint32_t)(w >> 32) & 3u;
      if (flag == kFlagPrefix) {
        excl += (uint32_t)w;
        break;
      }
      if (flag == kFlagAgg) {
        excl += (uint32_t)w;
        // j stops at 0 at the latest: tile 0 publishes only prefixes, and
        // if it publishes nothing the wait runs out at j = 0
        --j;
        spins = 0;
        continue;
      }
    }
    if (++spins > kSpinLimit) {
      atomicOr(err, kErrTimeout);
      break;
    }
  }
  store_status(status + tile, pack_status(epoch, kFlagPrefix, excl + agg));
  return excl;
}

// ------------------------------------------------------------- histogram

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint64_t* __restrict__ keys,
                                                            const unsigned long long* d_count,
                                                            PassPlan plan, uint32_t* ghist) {
  __shared__ uint32_t h[kMaxPasses][kRadixMax];
  for (int i = threadIdx.x; i < kMaxPasses * kRadixMax; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint64_t count = *d_count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint64_t x = __ldcs(keys + i);
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
      if (p < plan.passes) atomicAdd(&h[p][plan.digit(p, x)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < plan.passes * kRadixMax; i += blockDim.x) {
    uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// In-place exclusive scan of each pass's kRadixMax counts (one block per pass,
// kRadixMax / kSortThreads consecutive counts per thread).
__global__ void __launch_bounds__(kSortThreads) k_hist_scan(uint32_t* ghist) {
  constexpr int kPer = kRadixMax / kSortThreads;
  __shared__ uint32_t ws[kWarps];
  uint32_t* h = ghist + blockIdx.x * kRadixMax + threadIdx.x * kPer;
  uint32_t c[kPer], sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    c[q] = h[q];
    sum += c[q];
  }
  uint32_t total;
  uint32_t e = block_exclusive_scan(sum, ws, &total);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    h[q] = e;
    e += c[q];
  }
}

// ------------------------------------------------- duplicate filter + HLL

constexpr int kFilterItems = 8;  // keys per thread per tile

// Keys in[0, *d_in) pass through a device-wide direct-mapped cache of keys
// already kept (gcache, gmask + 1 slots; nullptr = keep every key): a key
// found there is dropped, since the thread that put it there keeps that copy;
// a key not found is kept and enters the cache at one in 2^admit of its
// positions.  Kept keys are compacted to out (one atomicAdd on *d_out per
// tile) and update the HyperLogLog registers (Flajolet, Fusy, Gandouet,
// Meunier 2007): register = top kHllBits bits of the mixed key, value = the
// position of the first one bit below them.  The cache entries of a thread's
// kFilterItems keys are read together, so their loads overlap.
__global__ void __launch_bounds__(kSortThreads) k_filter_hll(
    const uint64_t* __restrict__ in, const unsigned long long* d_in, uint64_t* __restrict__ out,
    unsigned long long* d_out, unsigned long long* gcache, uint32_t gmask, int admit,
    uint32_t* __restrict__ ghll) {
  constexpr uint64_t kTile = (uint64_t)kSortThreads * kFilterItems;
  __shared__ uint32_t reg[kHllRegs];
  __shared__ uint32_t ws[kWarps];
  __shared__ unsigned long long s_base;
  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  for (int i = tid; i < kHllRegs; i += kSortThreads) reg[i] = 0;
  __syncthreads();
  const uint64_t count = *d_in;
  const uint64_t tiles = (count + kTile - 1) / kTile;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t base = t * kTile + (uint64_t)w * 32 * kFilterItems;
    uint64_t k[kFilterItems];
    unsigned long long gv[kFilterItems];
#pragma unroll
    for (int i = 0; i < kFilterItems; ++i) {
      const uint64_t j = base + (uint64_t)i * 32 + lane;
      k[i] = j < count ? __ldcs(in + j) : 0ull;
    }
#pragma unroll
    for (int i = 0; i < kFilterItems; ++i) {
      const uint64_t j = base + (uint64_t)i * 32 + lane;
      gv[i] = (j < count && gcache != nullptr) ? __ldcg(gcache + ((uint32_t)(k[i] >> 20) & gmask))
                                               : 0ull;
    }
    uint32_t keep = 0;
#pragma unroll
    for (int i = 0; i < kFilterItems; ++i) {
      const uint64_t j = base + (uint64_t)i * 32 + lane;
      if (j >= count || (gcache != nullptr && gv[i] == k[i])) continue;
      keep |= 1u << i;
      if (gcache != nullptr && (admit == 0 || ((j * kGamma) >> (64 - admit)) == 0))
        __stcg(gcache + ((uint32_t)(k[i] >> 20) & gmask), (unsigned long long)k[i]);
      const uint64_t rest = k[i] << kHllBits;
      const uint32_t rank =
          rest ? (uint32_t)__clzll((long long)rest) + 1u : (uint32_t)(65 - kHllBits);
      atomicMax(&reg[(uint32_t)(k[i] >> (64 - kHllBits))], rank);
    }
    // warp totals, then one block scan over them; a warp writes the kept
    // keys of each item position as one contiguous run (coalesced stores)
    uint32_t wtot = 0;
#pragma unroll
    for (int i = 0; i < kFilterItems; ++i) wtot += __popc(__ballot_sync(kFull, (keep >> i) & 1u));
    if (lane == 0) ws[w] = wtot;
    __syncthreads();
    if (tid == 0) {
      uint32_t run = 0;
      for (int q = 0; q < kWarps; ++q) {
        const uint32_t c = ws[q];
        ws[q] = run;
        run += c;
      }
      s_base = run ? atomicAdd(d_out, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    uint64_t pos = s_base + ws[w];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kFilterItems; ++i) {
      const unsigned b = __ballot_sync(kFull, (keep >> i) & 1u);
      if ((keep >> i) & 1u) __stcs(out + pos + __popc(b & lt), k[i]);
      pos += __popc(b);
    }
    __syncthreads();
  }
  for (int i = tid; i < kHllRegs; i += kSortThreads)
    if (reg[i]) atomicMax(&ghll[i], reg[i]);
}

// ------------------------------------------------------------ one pass

// Digit-parallel look-back for the digits this thread owns: publish each
// digit's tile count as an aggregate, walk back over the preceding tiles until
// an inclusive prefix is found (all owned digits advance together, one load
// each per step), publish the inclusive prefixes.  Returns false if a bounded
// wait gave up.  A tile whose wait gave up still publishes what it summed as
// its inclusive prefix: that value is only a lower bound, so the tiles behind
// it compute offsets that are too low (their writes stay inside the output,
// which is bounds-checked) and the host, which sees kErrTimeout first,
// discards the whole phase.
template <int kPer>
__device__ __forceinline__ bool look_back_digits(uint64_t* status, uint32_t tile, int stride,
                                                 const uint32_t* dig, const uint32_t* cnt,
                                                 uint32_t* prefix, uint32_t epoch,
                                                 uint32_t spin_limit) {
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    prefix[q] = 0;
    store_status(status + (uint64_t)tile * stride + dig[q],
                 pack_status(epoch, tile == 0 ? kFlagPrefix : kFlagAgg, cnt[q]));
  }
  if (tile == 0) return true;
  uint32_t j[kPer];
  bool done[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    j[q] = tile - 1;
    done[q] = false;
  }
  bool ok = true;
  uint32_t spins = 0;
  for (;;) {
    bool all = true;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (done[q]) continue;
      uint64_t wd = load_status(status + (uint64_t)j[q] * stride + dig[q]);
      if ((uint32_t)(wd >> 34) == epoch) {
        uint32_t flag = (uint32_t)(wd >> 32) & 3u;
        if (flag == kFlagPrefix) {
          prefix[q] += (uint32_t)wd;
          done[q] = true;
          continue;
        }
        if (flag == kFlagAgg) {
          prefix[q] += (uint32_t)wd;
          // j stops at 0 at the latest: tile 0 publishes only prefixes, and
          // when it publishes nothing (the stall hook) this wait runs out at
          // j = 0 instead of moving past it
          --j[q];
          spins = 0;
        }
      }
      all = false;
    }
    if (all) break;
    if (++spins > spin_limit) {
      ok = false;
      break;
    }
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    store_status(status + (uint64_t)tile * stride + dig[q],
                 pack_status(epoch, kFlagPrefix, prefix[q] + cnt[q]));
  return ok;
}

// One stable counting pass over a 4096-key tile with 2^kRB digit values.
// Lanes holding the same digit are found by slicing the digit into bits and
// intersecting ballots (one vote per digit bit), so ranking needs no match
// instruction; each warp counts its digits in its own shared-memory row.
// Thread t owns digits t*kPer .. t*kPer+kPer-1 for the tile totals,
// look-back and scan.
template <int kRB>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_pass(
    const uint64_t* __restrict__ in, uint64_t* __restrict__ out, const unsigned long long* d_count,
    DigitFn dg, int bits, const uint32_t* __restrict__ digit_offset, uint64_t* status,
    uint32_t epoch, unsigned* ticket, unsigned* err, uint32_t* mark_flags, int half_bits,
    uint32_t spin_limit, int stall) {
  constexpr int kR = 1 << kRB;
  constexpr int kPer = kR / kSortThreads;
  extern __shared__ __align__(16) uint64_t sort_smem[];
  uint64_t* sk = sort_smem;                                              // [kSortTile]
  uint32_t(*whist)[kR] = reinterpret_cast<uint32_t(*)[kR]>(sk + kSortTile);  // [kWarps][kR]
  uint32_t* gofs = reinterpret_cast<uint32_t*>(whist + kWarps);            // [kR]
  __shared__ uint32_t ws[kWarps];
  __shared__ uint32_t s_tile;
  __shared__ int s_bad;

  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(ticket, 1u);
    s_bad = 0;
  }
  for (int i = tid; i < kWarps * kR; i += kSortThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  // test hook: tile 0 never publishes, so the waits behind it run out
  if (stall && tile == 0) return;
  const uint64_t count = *d_count;
  const uint64_t base = (uint64_t)tile * kSortTile;
  if (base >= count) return;
  const uint32_t nvalid =
      (uint32_t)(count - base < (uint64_t)kSortTile ? count - base : (uint64_t)kSortTile);

  // warp w owns tile positions [w*32*kSortItems, (w+1)*32*kSortItems); item i
  // of lane l is position w*32*kSortItems + i*32 + l
  uint64_t k[kSortItems];
  uint32_t off[kSortItems];
  const uint32_t wbase = w * 32 * kSortItems;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    uint32_t pos = wbase + i * 32 + lane;
    k[i] = pos < nvalid ? __ldcs(in + base + pos) : 0ull;
  }
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const bool valid = wbase + i * 32 + lane < nvalid;
    const uint32_t d = dg(k[i]);
    unsigned peers = __ballot_sync(kFull, valid);
#pragma unroll
    for (int b = 0; b < kRB; ++b) {
      if (b < bits) {
        unsigned v = __ballot_sync(kFull, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? v : ~v;
      }
    }
    uint32_t r = __popc(peers & lt);
    int leader = valid ? __ffs(peers) - 1 : (int)lane;
    uint32_t cnt = (valid && r == 0) ? whist[w][d] : 0u;
    cnt = __shfl_sync(kFull, cnt, leader);
    off[i] = cnt + r;
    if (valid && r == 0) whist[w][d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // per owned digit: prefix over warps, tile count, look-back
  uint32_t dig[kPer], tcount[kPer], prefix[kPer];
  uint32_t mine = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    dig[q] = tid * kPer + q;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      uint32_t t = whist[ww][dig[q]];
      whist[ww][dig[q]] = run;
      run += t;
    }
    tcount[q] = run;
    mine += run;
  }
  if (!look_back_digits<kPer>(status, tile, kR, dig, tcount, prefix, epoch, spin_limit)) {
    atomicOr(err, kErrTimeout);
    s_bad = 1;
  }
  uint32_t total;
  uint32_t tstart = block_exclusive_scan(mine, ws, &total);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) whist[ww][dig[q]] += tstart;
    gofs[dig[q]] = digit_offset[dig[q]] + prefix[q] - tstart;
    tstart += tcount[q];
  }
  __syncthreads();
  if (s_bad) return;  // offsets unknown: write nothing (the host sees kErrTimeout)

  // stage the tile in digit order
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (wbase + i * 32 + lane < nvalid) {
      const uint32_t at = whist[w][dg(k[i])] + off[i];
      if (index_ok(err, kKSortPass, at, nvalid)) sk[at] = k[i];
    }
  }
  __syncthreads();

  // coalesced write-out; optionally mark both endpoints of every key that
  // starts a run of equal keys inside the tile (the full-sort path)
  const uint64_t half_mask = (half_bits >= 64) ? ~0ull : ((1ull << half_bits) - 1);
  for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
    uint64_t key = sk[j];
    uint64_t gpos = (uint64_t)gofs[dg(key)] + j;
    if (gpos < count) __stcs(out + gpos, key);
    if (mark_flags != nullptr && (j == 0 || sk[j - 1] != key)) {
      mark_flag(mark_flags, key >> half_bits);
      mark_flag(mark_flags, key & half_mask);
    }
  }
}

// --------------------------------------------- hashed buckets and dedup

// bounds[b] = first position whose bucket is >= b, for b in [0, nb]; the
// mixed keys are partitioned in ascending order of their bucket (top hb bits).
__global__ void k_bucket_bounds(const uint64_t* __restrict__ keys,
                                const unsigned long long* d_count, int hb, uint32_t nb,
                                uint32_t* __restrict__ bounds) {
  const uint64_t count = *d_count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += stride) {
    uint64_t lo = 0, hi = count;
    while (lo < hi) {
      uint64_t mid = (lo + hi) >> 1;
      if (bucket_of(keys[mid], hb) < b) lo = mid + 1;
      else hi = mid;
    }
    bounds[b] = (uint32_t)lo;
  }
}

constexpr int kTableSlots = 2 * kBucketTarget;  // per-bucket shared-memory hash set (32 KB)
constexpr uint64_t kEmpty = ~0ull;  // never a mixed key (static_assert in lc_common.cuh)

// Insert into the open-addressing set with one compare-and-swap per probe
// (it also returns what the slot holds, so no separate read is needed);
// returns the slot when this call put the key there (a new distinct key),
// else -1.  *over is set when the table is full.
__device__ __forceinline__ int set_insert(uint64_t* table, uint64_t key, int* over) {
  uint32_t slot = (uint32_t)key & (kTableSlots - 1);  // low bits of the mixed key
  for (int probe = 0; probe < kTableSlots; ++probe) {
    uint64_t prev = atomicCAS((unsigned long long*)&table[slot], kEmpty, key);
    if (prev == kEmpty) return (int)slot;
    if (prev == key) return -1;
    slot = (slot + 1) & (kTableSlots - 1);
  }
  *over = 1;
  return -1;
}

// One bucket per iteration (claimed by ticket): insert its keys into a
// shared-memory open-addressing set (eight independent loads in flight per
// thread); each new distinct key also records its slot in a list, so the
// collection walks the list (about 2048 entries) instead of all table slots.
// The distinct keys are appended to `out` (one atomicAdd per bucket), both
// endpoints of each are marked in `flags`, and their slots are cleared.
__global__ void __launch_bounds__(kSortThreads) k_bucket_dedup(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ bounds, uint32_t nb,
    uint64_t* __restrict__ out, uint64_t cap, unsigned long long* m_next, uint32_t* flags,
    uint32_t n, int half_bits, unsigned* ticket, unsigned* err) {
  extern __shared__ __align__(16) uint64_t table[];  // [kTableSlots], then the slot list
  uint16_t* list = reinterpret_cast<uint16_t*>(table + kTableSlots);  // [kTableSlots]
  __shared__ uint32_t s_b, s_cnt;
  __shared__ unsigned long long s_base;
  __shared__ int s_over;
  const unsigned tid = threadIdx.x;
  constexpr int kIlp = 8;
  for (int i = tid; i < kTableSlots; i += kSortThreads) table[i] = kEmpty;
  if (tid == 0) s_over = 0;
  const uint64_t half_mask = (1ull << half_bits) - 1;
  for (;;) {
    if (tid == 0) {
      s_b = atomicAdd(ticket, 1u);
      s_cnt = 0;
    }
    __syncthreads();
    const uint32_t b = s_b;
    if (b >= nb) break;
    const uint32_t lo = bounds[b], hi = bounds[b + 1];
    for (uint32_t i0 = lo; i0 < hi; i0 += kSortThreads * kIlp) {
      uint64_t kk[kIlp];
#pragma unroll
      for (int j = 0; j < kIlp; ++j) {
        uint32_t i = i0 + j * kSortThreads + tid;
        kk[j] = i < hi ? __ldcs(keys + i) : kEmpty;
      }
#pragma unroll
      for (int j = 0; j < kIlp; ++j) {
        if (kk[j] == kEmpty) continue;
        const int slot = set_insert(table, kk[j], &s_over);
        if (slot >= 0) list[atomicAdd(&s_cnt, 1u)] = (uint16_t)slot;
      }
    }
    __syncthreads();
    const uint32_t total = s_cnt;
    if (tid == 0) {
      s_base = total ? atomicAdd(m_next, (unsigned long long)total) : 0ull;
      if (s_over) {
        atomicOr(err, kErrOverflow);
        s_over = 0;
      }
    }
    __syncthreads();
    for (uint32_t e = tid; e < total; e += kSortThreads) {
      const uint32_t slot = list[e];
      const uint64_t v = table[slot];
      const uint64_t pos = s_base + e;
      if (index_ok(err, kKBucketDedup, pos, cap)) out[pos] = v;
      const uint64_t k = key_unmix(v);
      const uint64_t a = k >> half_bits, c = k & half_mask;
      if (index_ok(err, kKBucketDedup, a > c ? a : c, n)) {
        mark_flag(flags, a);
        mark_flag(flags, c);
      }
      table[slot] = kEmpty;
    }
    // the next iteration's barrier orders these clears before new inserts
  }
}

// e[j] = (id(a) << 32 | id(b)) for e[j] = key_mix(a << half_bits | b), id the
// keep rank.
__global__ void k_rename(uint64_t* __restrict__ e, const unsigned long long* d_count,
                         uint64_t cap, int half_bits, const uint64_t* __restrict__ rank,
                         uint32_t n, unsigned* err) {
  const uint64_t count = *d_count;
  if (!index_ok(err, kKRename, count, cap + 1)) return;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t half_mask = (1ull << half_bits) - 1;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
    uint64_t k = key_unmix(e[j]);
    const uint64_t a = k >> half_bits, b = k & half_mask;
    if (!index_ok(err, kKRename, a > b ? a : b, n)) continue;
    uint32_t ia, ib;
    keep_rank(rank, (uint32_t)a, &ia);
    keep_rank(rank, (uint32_t)b, &ib);
    e[j] = ((uint64_t)ia << 32) | ib;
  }
}

// In place: e[j] = key_unmix(e[j]) (before the full-sort fallback).
__global__ void k_unmix(uint64_t* __restrict__ e, const unsigned long long* d_count) {
  const uint64_t count = *d_count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride)
    e[j] = key_unmix(e[j]);
}

// ------------------------------------------------------------- scans

constexpr int kScanItems = 16;
constexpr int kScanTile = kSortThreads * kScanItems;
constexpr int kRankItems = 4;  // flag words per thread
constexpr int kRankTile = kSortThreads * kRankItems;

// Keep ranks (rank_words) from the flag bitmap, by a single-pass scan of the
// words' popcounts with decoupled look-back; each kept node's mo value is
// copied to its new id.
__global__ void __launch_bounds__(kSortThreads) k_scan_flags(
    const uint32_t* __restrict__ flags, uint64_t* __restrict__ rank, uint32_t n,
    const uint32_t* __restrict__ mo_in, uint32_t* __restrict__ mo_out,
    unsigned long long* total_out, uint64_t* status, uint32_t epoch, unsigned* ticket,
    unsigned* err) {
  __shared__ uint32_t ws[kWarps];
  __shared__ uint32_t s_tile, s_excl;
  const unsigned tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t nw = rank_words(n), fw = flag_words(n);
  const uint64_t base = (uint64_t)tile * kRankTile;
  if (base >= nw) return;
  const uint64_t w0 = base + (uint64_t)tid * kRankItems;
  uint32_t f[kRankItems];
  if (w0 + kRankItems <= fw) {
    const uint4 q = *reinterpret_cast<const uint4*>(flags + w0);
    f[0] = q.x; f[1] = q.y; f[2] = q.z; f[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < kRankItems; ++i) f[i] = w0 + i < fw ? flags[w0 + i] : 0u;
  }
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < kRankItems; ++i) sum += __popc(f[i]);
  uint32_t tile_total;
  const uint32_t e = block_exclusive_scan(sum, ws, &tile_total);
  if (tid == 0) s_excl = look_back(status, tile, tile_total, epoch, err);
  __syncthreads();
  uint32_t run = s_excl + e;
#pragma unroll
  for (int i = 0; i < kRankItems; ++i) {
    if (w0 + i < nw) rank[w0 + i] = ((uint64_t)run << 32) | f[i];
    if (mo_out != nullptr) {
      uint32_t bits = f[i], r = run;
      while (bits) {
        const uint64_t v = 32 * (w0 + i) + (uint32_t)(__ffs(bits) - 1);
        if (index_ok(err, kKScanFlags, v, n)) mo_out[r] = mo_in[v];
        ++r;
        bits &= bits - 1u;
      }
    }
    run += __popc(f[i]);
  }
  if (base + kRankTile >= nw && tid == 0) *total_out = s_excl + tile_total;
}

__global__ void __launch_bounds__(kSortThreads) k_unique_rename(
    const uint64_t* __restrict__ keys, const unsigned long long* d_count, int half_bits,
    const uint64_t* __restrict__ rank, uint32_t n, uint64_t* __restrict__ out,
    unsigned long long* m_next, uint64_t* status, uint32_t epoch, unsigned* ticket,
    unsigned* err) {
  __shared__ uint32_t ws[kWarps];
  __shared__ uint32_t s_tile, s_excl;
  const unsigned tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t count = *d_count;
  const uint64_t base = (uint64_t)tile * kScanTile;
  if (base >= count) return;
  const uint64_t i0 = base + (uint64_t)tid * kScanItems;
  uint64_t k[kScanItems];
  uint32_t fl = 0;
  uint64_t prev = i0 > 0 && i0 - 1 < count ? keys[i0 - 1] : ~0ull;
  if (i0 + kScanItems <= count) {
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(keys + i0);
#pragma unroll
    for (int i = 0; i < kScanItems / 2; ++i) {
      ulonglong2 q = __ldcs(src + i);
      k[2 * i] = q.x;
      k[2 * i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) k[i] = i0 + i < count ? keys[i0 + i] : 0ull;
  }
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    bool valid = i0 + i < count;
    bool first = valid && k[i] != prev;
    fl |= (first ? 1u : 0u) << i;
    prev = k[i];
  }
  uint32_t tile_total;
  uint32_t e = block_exclusive_scan(__popc(fl), ws, &tile_total);
  if (tid == 0) s_excl = look_back(status, tile, tile_total, epoch, err);
  __syncthreads();
  uint64_t pos = (uint64_t)s_excl + e;
  const uint64_t half_mask = (1ull << half_bits) - 1;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (fl & (1u << i)) {
      const uint64_t ka = k[i] >> half_bits, kb = k[i] & half_mask;
      if (index_ok(err, kKUniqueRename, ka > kb ? ka : kb, n)) {
        uint32_t a, b;
        keep_rank(rank, (uint32_t)ka, &a);
        keep_rank(rank, (uint32_t)kb, &b);
        out[pos] = ((uint64_t)a << 32) | b;
      }
      ++pos;
    }
  }
  if (base + kScanTile >= count && tid == 0) *m_next = (unsigned long long)s_excl + tile_total;
}


// ------------------------------------------------- phase-0 edge buckets

struct EdgeBlocks {
  uint32_t scale, nb;
  __device__ __forceinline__ uint32_t blk(uint32_t v) const {
    return min(__umulhi(v, scale), nb - 1u);
  }
  __device__ __forceinline__ uint32_t digit(uint32_t u, uint32_t v) const {
    const uint32_t a = blk(u), b = blk(v);
    return min(a, b) * nb + max(a, b);
  }
};

constexpr int kBktItems = 8;
constexpr int kBktTile = kSortThreads * kBktItems;  // edges per tile

// Bucket counts of the input edges (ids >= n count as the loop (0, 0)).
__global__ void __launch_bounds__(kSortThreads) k_bucket_hist(
    const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m, uint32_t n,
    int vec, EdgeBlocks eb, uint32_t* __restrict__ ghist, unsigned* err) {
  __shared__ uint32_t h[kBucketMaxDigits];
  const uint32_t nd = eb.nb * eb.nb;
  for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) h[i] = 0;
  __syncthreads();
  bool bad = false;
  auto count = [&](uint32_t u, uint32_t v) {
    if (u >= n || v >= n) {
      bad = true;
      u = v = 0;
    }
    atomicAdd(&h[eb.digit(u, v)], 1u);
  };
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t done = 0;
  if (vec) {
    const uint64_t nq = m / 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const uint4* d4 = reinterpret_cast<const uint4*>(dst);
    for (uint64_t q = gt; q < nq; q += stride) {
      const uint4 a = __ldcs(s4 + q), b = __ldcs(d4 + q);
      count(a.x, b.x);
      count(a.y, b.y);
      count(a.z, b.z);
      count(a.w, b.w);
    }
    done = nq * 4;
  }
  for (uint64_t j = done + gt; j < m; j += stride) count(__ldcs(src + j), __ldcs(dst + j));
  if (bad) atomicOr(err, kErrBadVertex);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x)
    if (h[i]) atomicAdd(&ghist[i], h[i]);
}

// fill[d * kBucketFillStride] = first position of bucket d (exclusive scan of
// the counts; one block, four buckets per thread).
__global__ void __launch_bounds__(kSortThreads) k_bucket_starts(const uint32_t* __restrict__ ghist,
                                                                uint32_t nd, uint32_t* fill) {
  __shared__ uint32_t ws[kWarps];
  constexpr int kPer = kBucketMaxDigits / kSortThreads;
  uint32_t c[kPer], sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const uint32_t d = threadIdx.x * kPer + q;
    c[q] = d < nd ? ghist[d] : 0u;
    sum += c[q];
  }
  uint32_t total;
  uint32_t e = block_exclusive_scan(sum, ws, &total);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const uint32_t d = threadIdx.x * kPer + q;
    if (d < nd) fill[d * kBucketFillStride] = e;
    e += c[q];
  }
}

// Scatter of the input edges into their buckets.  Order inside a bucket does
// not matter, so a tile of kBktTile edges is ranked with shared-memory
// atomics (no stable ranking, no look-back): each bucket's tile count is
// reserved in the bucket with one global atomicAdd on its fill counter (the
// counters sit one cache line apart), the tile is staged in shared memory in
// bucket order and written out in runs.
__global__ void __launch_bounds__(kSortThreads) k_bucket_scatter(
    const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m, uint32_t n,
    int vec, EdgeBlocks eb, uint32_t* fill, uint64_t* __restrict__ out, unsigned* err) {
  __shared__ uint64_t stage[kBktTile];
  __shared__ uint32_t s_cnt[kBucketMaxDigits];
  __shared__ uint32_t s_off[kBucketMaxDigits];
  __shared__ uint32_t s_gb[kBucketMaxDigits];
  __shared__ uint32_t ws[kWarps];
  constexpr int kPer = kBucketMaxDigits / kSortThreads;
  const unsigned tid = threadIdx.x;
  const uint32_t nd = eb.nb * eb.nb;
  for (uint32_t i = tid; i < nd; i += kSortThreads) s_cnt[i] = 0;
  __syncthreads();
  const uint64_t ntiles = (m + kBktTile - 1) / kBktTile;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = t * kBktTile;
    uint32_t u[kBktItems], v[kBktItems];
    if (vec && base + kBktTile <= m) {
      // item 4*i + c is edge base + 4 * (i * kSortThreads + tid) + c
      const uint4* s4 = reinterpret_cast<const uint4*>(src + base);
      const uint4* d4 = reinterpret_cast<const uint4*>(dst + base);
#pragma unroll
      for (int i = 0; i < kBktItems / 4; ++i) {
        const uint4 a = __ldcs(s4 + i * kSortThreads + tid), b = __ldcs(d4 + i * kSortThreads + tid);
        u[4 * i] = a.x; u[4 * i + 1] = a.y; u[4 * i + 2] = a.z; u[4 * i + 3] = a.w;
        v[4 * i] = b.x; v[4 * i + 1] = b.y; v[4 * i + 2] = b.z; v[4 * i + 3] = b.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kBktItems; ++i) {
        const uint64_t j = base + (uint64_t)i * kSortThreads + tid;
        u[i] = j < m ? __ldcs(src + j) : 0u;
        v[i] = j < m ? __ldcs(dst + j) : 0u;
      }
    }
    const uint32_t nvalid = (uint32_t)(m - base < (uint64_t)kBktTile ? m - base : (uint64_t)kBktTile);
    // per item: bucket << 16 | rank inside the tile's run of that bucket
    // (bucket 0xFFFF: not an item)
    uint32_t dr[kBktItems];
#pragma unroll
    for (int i = 0; i < kBktItems; ++i) {
      // every item of a full tile is valid; in the last tile the first nvalid
      // positions are, whichever load form was used (the vector form needs a
      // full tile)
      const uint32_t pos = (vec && base + kBktTile <= m)
                               ? 4u * ((i >> 2) * kSortThreads + tid) + (i & 3)
                               : (uint32_t)i * kSortThreads + tid;
      if (pos < nvalid) {
        if (u[i] >= n || v[i] >= n) u[i] = v[i] = 0;  // reported by k_bucket_hist
        const uint32_t d = eb.digit(u[i], v[i]);
        dr[i] = (d << 16) | atomicAdd(&s_cnt[d], 1u);
      } else {
        dr[i] = 0xFFFF0000u;
      }
    }
    __syncthreads();
    // in-tile bucket offsets, and the tile's range in every bucket it feeds
    uint32_t c[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const uint32_t d = tid * kPer + q;
      c[q] = d < nd ? s_cnt[d] : 0u;
      sum += c[q];
    }
    uint32_t tot;
    uint32_t e = block_exclusive_scan(sum, ws, &tot);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const uint32_t d = tid * kPer + q;
      if (d < nd) {
        s_off[d] = e;
        if (c[q]) s_gb[d] = atomicAdd(&fill[d * kBucketFillStride], c[q]);
      }
      e += c[q];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kBktItems; ++i) {
      if ((dr[i] >> 16) < nd) {
        const uint32_t at = s_off[dr[i] >> 16] + (dr[i] & 0xFFFFu);
        if (index_ok(err, kKBucketEdges, at, nvalid))
          stage[at] = ((uint64_t)u[i] << 32) | v[i];
      }
    }
    __syncthreads();
    for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
      const uint64_t x = stage[j];
      const uint32_t d = eb.digit((uint32_t)(x >> 32), (uint32_t)x);
      const uint64_t pos = (uint64_t)s_gb[d] + (j - s_off[d]);
      if (index_ok(err, kKBucketEdges, pos, m)) out[pos] = x;
    }
    __syncthreads();
    for (uint32_t i = tid; i < nd; i += kSortThreads) s_cnt[i] = 0;
    __syncthreads();
  }
}


// ------------------------------------------------ segmented deduplication

constexpr int kSegFilterThreads = 512;
constexpr int kSegFilterItems = 8;
constexpr int kSegFilterTile = kSegFilterThreads * kSegFilterItems;
constexpr int kSegInsItems = 8;
constexpr int kSegInsTile = kSortThreads * kSegInsItems;

__device__ __forceinline__ uint32_t seg_of(uint64_t y) { return (uint32_t)(y >> (64 - kSegBits)); }

// starts[s] = exclusive scan of the per-segment key counts scratch[0, kSegs);
// the fill counters start at the starts.
__global__ void __launch_bounds__(kSortThreads) k_seg_starts(uint32_t* scratch) {
  static_assert(kSegs == kSortThreads, "one segment per thread");
  __shared__ uint32_t ws[kWarps];
  const uint32_t c = scratch[threadIdx.x];
  uint32_t total;
  const uint32_t e = block_exclusive_scan(c, ws, &total);
  scratch[kSegStartOff + threadIdx.x] = e;
  scratch[kBucketMaxDigits + threadIdx.x * kBucketFillStride] = e;
  if (threadIdx.x == 0) scratch[kSegStartOff + kSegs] = total;
}

// k_filter_hll whose kept keys go to their segment's region: a tile's kept
// keys are ranked per segment in shared memory, each segment's share is
// reserved with one atomicAdd on its fill counter, and the tile is staged in
// segment order and written out in runs.
__global__ void __launch_bounds__(kSegFilterThreads) k_filter_seg(
    const uint64_t* __restrict__ in, const unsigned long long* d_in, uint64_t* __restrict__ out,
    uint64_t cap, unsigned long long* d_out, unsigned long long* gcache, uint32_t gmask, int admit,
    uint32_t* __restrict__ ghll, uint32_t* scratch, unsigned* err) {
  __shared__ uint32_t reg[kHllRegs];
  __shared__ uint64_t stage[kSegFilterTile];
  __shared__ uint32_t s_cnt[kSegs], s_off[kSegs], s_gb[kSegs];
  __shared__ uint32_t ws[kSegFilterThreads / 32];
  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  uint32_t* fill = scratch + kBucketMaxDigits;
  for (int i = tid; i < kHllRegs; i += kSegFilterThreads) reg[i] = 0;
  if (tid < kSegs) s_cnt[tid] = 0;
  __syncthreads();
  const uint64_t count = *d_in;
  const uint64_t tiles = (count + kSegFilterTile - 1) / kSegFilterTile;
  unsigned long long kept_total = 0;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t base = t * kSegFilterTile + (uint64_t)w * 32 * kSegFilterItems;
    uint64_t k[kSegFilterItems];
    unsigned long long gv[kSegFilterItems];
#pragma unroll
    for (int i = 0; i < kSegFilterItems; ++i) {
      const uint64_t j = base + (uint64_t)i * 32 + lane;
      k[i] = j < count ? __ldcs(in + j) : 0ull;
    }
#pragma unroll
    for (int i = 0; i < kSegFilterItems; ++i) {
      const uint64_t j = base + (uint64_t)i * 32 + lane;
      gv[i] = (j < count && gcache != nullptr) ? __ldcg(gcache + ((uint32_t)(k[i] >> 20) & gmask))
                                               : 0ull;
    }
    uint32_t dr[kSegFilterItems];
#pragma unroll
    for (int i = 0; i < kSegFilterItems; ++i) {
      const uint64_t j = base + (uint64_t)i * 32 + lane;
      dr[i] = 0xFFFF0000u;
      if (j >= count || (gcache != nullptr && gv[i] == k[i])) continue;
      if (gcache != nullptr && (admit == 0 || ((j * kGamma) >> (64 - admit)) == 0))
        __stcg(gcache + ((uint32_t)(k[i] >> 20) & gmask), (unsigned long long)k[i]);
      const uint64_t rest = k[i] << kHllBits;
      const uint32_t rank =
          rest ? (uint32_t)__clzll((long long)rest) + 1u : (uint32_t)(65 - kHllBits);
      atomicMax(&reg[(uint32_t)(k[i] >> (64 - kHllBits))], rank);
      const uint32_t d = seg_of(k[i]);
      dr[i] = (d << 16) | atomicAdd(&s_cnt[d], 1u);
    }
    __syncthreads();
    const uint32_t c = tid < kSegs ? s_cnt[tid] : 0u;
    uint32_t tot;
    const uint32_t e = block_exclusive_scan<kSegFilterThreads>(c, ws, &tot);
    if (tid < kSegs) {
      s_off[tid] = e;
      if (c) s_gb[tid] = atomicAdd(&fill[tid * kBucketFillStride], c);
    }
    kept_total += tot;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSegFilterItems; ++i) {
      if ((dr[i] >> 16) < kSegs) {
        const uint32_t at = s_off[dr[i] >> 16] + (dr[i] & 0xFFFFu);
        if (index_ok(err, kKSegDedup, at, tot)) stage[at] = k[i];
      }
    }
    __syncthreads();
    for (uint32_t j = tid; j < tot; j += kSegFilterThreads) {
      const uint64_t x = stage[j];
      const uint32_t d = seg_of(x);
      const uint64_t pos = (uint64_t)s_gb[d] + (j - s_off[d]);
      if (index_ok(err, kKSegDedup, pos, cap)) __stcg(out + pos, x);
    }
    __syncthreads();
    if (tid < kSegs) s_cnt[tid] = 0;
    __syncthreads();
  }
  if (tid == 0 && kept_total) atomicAdd(d_out, kept_total);
  for (int i = tid; i < kHllRegs; i += kSegFilterThreads)
    if (reg[i]) atomicMax(&ghll[i], reg[i]);
}

// tile prefix of the segments: tiles[s] = sum over earlier segments of
// ceil(kept_s / kSegInsTile), kept_s = fill_s - start_s.
__global__ void __launch_bounds__(kSortThreads) k_seg_tiles(uint32_t* scratch) {
  __shared__ uint32_t ws[kWarps];
  const uint32_t s = threadIdx.x;
  const uint32_t kept = scratch[kBucketMaxDigits + s * kBucketFillStride] - scratch[kSegStartOff + s];
  const uint32_t nt = (kept + kSegInsTile - 1) / kSegInsTile;
  uint32_t total;
  const uint32_t e = block_exclusive_scan(nt, ws, &total);
  scratch[kSegTileOff + s] = e;
  if (s == 0) scratch[kSegTileOff + kSegs] = total;
}

// Distinct keys of segments [seg_lo, seg_hi): tiles claimed in order by
// ticket (so the tiles in flight stay within a segment or two and their
// slices stay in L2; a fixed tile-to-block assignment lets the blocks drift
// apart until the slices in use no longer fit); a key probes its segment's
// slice (slots entries, linear probing from its low bits) with a read
// through L2 and, on an empty slot, a compare-and-swap.  Slots only ever
// change from empty to a key, so a read that returns the key itself settles
// the probe, and a stale empty only costs the compare-and-swap.  Keys new to the table are staged per tile,
// appended to `out` with one atomicAdd per tile, and both endpoints of each
// are marked in flags.  A slice that fills up raises kErrOverflow.
__global__ void __launch_bounds__(kSortThreads) k_seg_insert(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ scratch, uint32_t seg_lo,
    uint32_t seg_hi, uint64_t slots, unsigned long long* table, uint64_t* __restrict__ out,
    uint64_t cap, unsigned long long* m_next, uint32_t* flags, uint32_t n, int half_bits,
    unsigned* ticket, unsigned* err) {
  __shared__ uint64_t fresh[kSegInsTile];
  __shared__ uint32_t s_new, s_t;
  __shared__ unsigned long long s_base;
  const unsigned tid = threadIdx.x;
  const uint32_t* tiles = scratch + kSegTileOff;
  const uint32_t* starts = scratch + kSegStartOff;
  const uint32_t* fill = scratch + kBucketMaxDigits;
  const uint32_t t0 = tiles[seg_lo], t1 = tiles[seg_hi];
  const uint64_t half_mask = (1ull << half_bits) - 1;
  const uint64_t smask = slots - 1;
  // thread 0 claims the next tile while this one is processed (the claim's
  // round trip is hidden) and publishes it after the tile's closing barrier
  uint32_t next_t = 0;
  if (tid == 0) {
    s_new = 0;
    s_t = t0 + atomicAdd(ticket, 1u);
  }
  __syncthreads();
  for (;;) {
    const uint32_t t = s_t;
    if (t >= t1) break;
    if (tid == 0) next_t = t0 + atomicAdd(ticket, 1u);
    // segment of tile t: last s in [seg_lo, seg_hi) with tiles[s] <= t
    uint32_t lo = seg_lo, hi = seg_hi - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (tiles[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const uint32_t sg = lo;
    const uint64_t kb = (uint64_t)starts[sg] + (uint64_t)(t - tiles[sg]) * kSegInsTile;
    const uint64_t ke = fill[sg * kBucketFillStride];
    unsigned long long* slice = table + (uint64_t)(sg - seg_lo) * slots;
    uint64_t k[kSegInsItems];
#pragma unroll
    for (int i = 0; i < kSegInsItems; ++i) {
      const uint64_t j = kb + (uint64_t)i * kSortThreads + tid;
      k[i] = (j < ke && j < cap) ? __ldcs(keys + j) : kEmpty;
    }
#pragma unroll
    for (int i = 0; i < kSegInsItems; ++i) {
      if (k[i] == kEmpty) continue;
      uint64_t slot = k[i] & smask;
      bool done = false;
      for (uint64_t probe = 0; probe < slots; ++probe) {
        const unsigned long long cur = __ldcg(slice + slot);
        if (cur == k[i]) {
          done = true;
          break;
        }
        if (cur == kEmpty) {
          const unsigned long long old = atomicCAS(slice + slot, kEmpty, k[i]);
          if (old == kEmpty) {
            fresh[atomicAdd(&s_new, 1u)] = k[i];
            done = true;
            break;
          }
          if (old == k[i]) {
            done = true;
            break;
          }
        }
        slot = (slot + 1) & smask;
      }
      if (!done) atomicOr(err, kErrOverflow);
    }
    __syncthreads();
    const uint32_t nn = s_new;
    if (tid == 0) s_base = nn ? atomicAdd(m_next, (unsigned long long)nn) : 0ull;
    __syncthreads();
    for (uint32_t e = tid; e < nn; e += kSortThreads) {
      const uint64_t v = fresh[e];
      const uint64_t pos = s_base + e;
      if (index_ok(err, kKSegDedup, pos, cap)) out[pos] = v;
      const uint64_t kk = key_unmix(v);
      const uint64_t a = kk >> half_bits, b = kk & half_mask;
      if (index_ok(err, kKSegDedup, a > b ? a : b, n)) {
        mark_flag(flags, a);
        mark_flag(flags, b);
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_new = 0;
      s_t = next_t;
    }
    __syncthreads();
  }
}

// out[prefix of kept counts + j] = the j-th kept key of each segment.
__global__ void k_seg_compact(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ scratch,
                              uint64_t* __restrict__ out) {
  const uint32_t* starts = scratch + kSegStartOff;
  const uint32_t* fill = scratch + kBucketMaxDigits;
  __shared__ uint64_t s_dst;
  for (uint32_t sg = blockIdx.x; sg < kSegs; sg += gridDim.x) {
    if (threadIdx.x == 0) {
      uint64_t before = 0;
      for (uint32_t q = 0; q < sg; ++q) before += fill[q * kBucketFillStride] - starts[q];
      s_dst = before;
    }
    __syncthreads();
    const uint64_t b = starts[sg], e = fill[sg * kBucketFillStride];
    for (uint64_t j = b + threadIdx.x; j < e; j += blockDim.x) out[s_dst + (j - b)] = keys[j];
    __syncthreads();
  }
}

}  // namespace

// ------------------------------------------------------------- host side

uint32_t bucket_blocks_for(uint32_t n, uint64_t window_bytes) {
  const uint64_t w = std::max<uint64_t>(window_bytes, 1);
  const uint64_t nb = (16ull * n + w - 1) / w;
  return (uint32_t)std::min<uint64_t>(kBucketMaxBlocks, std::max<uint64_t>(2, nb));
}

// scale = ceil(nb * 2^32 / n); blocks are clamped to nb - 1 (needs n >= nb)
static EdgeBlocks edge_blocks(uint32_t n, uint32_t* nb) {
  *nb = std::max<uint32_t>(2, std::min(*nb, kBucketMaxBlocks));
  const uint64_t sc = (((uint64_t)*nb << 32) + n - 1) / std::max<uint32_t>(n, *nb);
  return EdgeBlocks{(uint32_t)std::min<uint64_t>(sc, 0xFFFFFFFFull), *nb};
}

static int both_aligned16(const uint32_t* src, const uint32_t* dst) {
  return ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
}

void bucket_clear(uint32_t n, uint32_t nb, uint32_t* scratch, const Launch& L) {
  edge_blocks(n, &nb);
  cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * nb * nb, L.stream);
}

void bucket_count(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t nb,
                  uint32_t* scratch, unsigned* err, const Launch& L) {
  if (m == 0) return;
  const EdgeBlocks eb = edge_blocks(n, &nb);
  KScope ks(L, kKBucketEdges);
  const int hgrid = (int)std::min<uint64_t>((m + 4095) / 4096, (uint64_t)L.sms * 8);
  k_bucket_hist<<<hgrid, kSortThreads, 0, L.stream>>>(src, dst, m, n, both_aligned16(src, dst),
                                                      eb, scratch, err);
}

void bucket_edges(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t nb,
                  uint64_t* out, uint32_t* scratch, unsigned* err, const Launch& L) {
  if (m == 0) return;
  bucket_clear(n, nb, scratch, L);
  bucket_count(src, dst, m, n, nb, scratch, err, L);
  bucket_place(src, dst, m, n, nb, out, scratch, err, L);
}

void bucket_place(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t nb,
                  uint64_t* out, uint32_t* scratch, unsigned* err, const Launch& L) {
  if (m == 0) return;
  const EdgeBlocks eb = edge_blocks(n, &nb);
  const uint32_t nd = nb * nb;
  const int vec = both_aligned16(src, dst);
  uint32_t* hist = scratch;
  uint32_t* fill = scratch + kBucketMaxDigits;
  {
    KScope ks(L, kKBucketEdges);
    k_bucket_starts<<<1, kSortThreads, 0, L.stream>>>(hist, nd, fill);
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bucket_scatter, kSortThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int sgrid =
      (int)std::min<uint64_t>((m + kBktTile - 1) / kBktTile, (uint64_t)L.sms * per_sm);
  KScope ks(L, kKBucketEdges);
  k_bucket_scatter<<<sgrid, kSortThreads, 0, L.stream>>>(src, dst, m, n, vec, eb, fill, out, err);
}

// ---- tiles over chunk-local buckets

// Segment s = d * chunks + c is bucket d of chunk c (bucket order first, so
// the tiles of one vertex-block pair stay together).  One block: exclusive
// scan of the segments' tile counts into first[s] (first[segs] = total).
__global__ void __launch_bounds__(kSortThreads) k_chunk_tile_scan(
    const uint32_t* __restrict__ chunk_scratch, uint32_t chunks, uint32_t nd, uint32_t tile_edges,
    uint32_t* __restrict__ first, unsigned long long* ntiles) {
  __shared__ uint32_t ws[kWarps];
  const uint32_t segs = nd * chunks;
  uint32_t carry = 0;
  for (uint32_t s0 = 0; s0 < segs; s0 += kSortThreads) {
    const uint32_t s = s0 + threadIdx.x;
    uint32_t t = 0;
    if (s < segs) {
      const uint32_t d = s / chunks, c = s % chunks;
      const uint32_t cnt = chunk_scratch[(uint64_t)c * kChunkScratchWords + d];
      t = (cnt + tile_edges - 1) / tile_edges;
    }
    uint32_t tot;
    const uint32_t e = block_exclusive_scan(t, ws, &tot);
    if (s < segs) first[s] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    first[segs] = carry;
    *ntiles = carry;
  }
}

// One warp per segment writes its tiles' (first edge, end).
__global__ void k_chunk_tile_fill(const uint32_t* __restrict__ chunk_scratch, uint32_t chunks,
                                  uint32_t nd, uint64_t chunk, uint32_t tile_edges,
                                  const uint32_t* __restrict__ first, uint64_t* __restrict__ tiles,
                                  uint64_t max_tiles, unsigned* err) {
  const uint32_t segs = nd * chunks;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < segs; s += nw) {
    const uint32_t d = s / chunks, c = s % chunks;
    const uint32_t* cs = chunk_scratch + (uint64_t)c * kChunkScratchWords;
    const uint32_t cnt = cs[d];
    // after bucket_place, the fill counter of bucket d is its end in the chunk
    const uint64_t begin = (uint64_t)c * chunk + cs[kBucketMaxDigits + d * kBucketFillStride] - cnt;
    const uint32_t f = first[s], nt = first[s + 1] - f;
    for (uint32_t q = lane_id(); q < nt; q += 32) {
      const uint64_t b = begin + (uint64_t)q * tile_edges;
      const uint64_t e = b + tile_edges < begin + cnt ? b + tile_edges : begin + cnt;
      if (index_ok(err, kKBucketEdges, (uint64_t)f + q, max_tiles)) {
        tiles[2ull * (f + q)] = b;
        tiles[2ull * (f + q) + 1] = e;
      }
    }
  }
}

static uint64_t max_chunk_tiles(uint64_t m, uint32_t nd, uint32_t chunks, uint32_t tile_edges) {
  return m / tile_edges + (uint64_t)nd * chunks + 1;
}

uint64_t chunk_tiles_bytes(uint64_t m, uint32_t nb, uint32_t chunks, uint32_t tile_edges) {
  nb = std::max<uint32_t>(2, std::min(nb, kBucketMaxBlocks));
  const uint64_t nd = (uint64_t)nb * nb;
  return 16 * max_chunk_tiles(m, (uint32_t)nd, chunks, tile_edges) + 4 * (nd * chunks + 1);
}

void chunk_tiles(const uint32_t* chunk_scratch, uint32_t chunks, uint64_t chunk, uint64_t m,
                 uint32_t n, uint32_t nb, uint32_t tile_edges, uint64_t* tiles,
                 unsigned long long* ntiles, unsigned* err, const Launch& L) {
  edge_blocks(n, &nb);
  const uint32_t nd = nb * nb;
  // the segments' first tiles are kept behind the tiles (see chunk_tiles_bytes)
  const uint64_t max_tiles = max_chunk_tiles(m, nd, chunks, tile_edges);
  uint32_t* first = reinterpret_cast<uint32_t*>(tiles + 2 * max_tiles);
  KScope ks(L, kKBucketEdges);
  k_chunk_tile_scan<<<1, kSortThreads, 0, L.stream>>>(chunk_scratch, chunks, nd, tile_edges,
                                                      first, ntiles);
  const uint32_t segs = nd * chunks;
  const int grid = (int)std::min<uint64_t>((32ull * segs + kSortThreads - 1) / kSortThreads,
                                           (uint64_t)L.sms * 8);
  k_chunk_tile_fill<<<grid, kSortThreads, 0, L.stream>>>(chunk_scratch, chunks, nd, chunk,
                                                         tile_edges, first, tiles, max_tiles, err);
}

void seg_begin(uint32_t* scratch, const Launch& L) {
  KScope ks(L, kKSegDedup);
  k_seg_starts<<<1, kSortThreads, 0, L.stream>>>(scratch);
}

void filter_seg(const uint64_t* in, const unsigned long long* d_in, uint64_t max_count,
                uint64_t* out, unsigned long long* d_out, unsigned long long* gcache,
                uint32_t gslots, int admit, uint32_t* hll, uint32_t* scratch, unsigned* err,
                const Launch& L) {
  if (max_count == 0) return;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_seg, kSegFilterThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int grid = (int)std::min<uint64_t>((max_count + kSegFilterTile - 1) / kSegFilterTile,
                                           (uint64_t)L.sms * per_sm);
  KScope ks(L, kKFilter);
  k_filter_seg<<<grid, kSegFilterThreads, 0, L.stream>>>(in, d_in, out, max_count, d_out,
                                                    gslots ? gcache : nullptr,
                                                    gslots ? gslots - 1 : 0u, admit, hll, scratch,
                                                    err);
}

bool seg_dedup(const uint64_t* keys, uint32_t* scratch, uint64_t max_count, uint64_t* table,
               uint64_t table_slots, uint64_t slots, uint64_t* out, unsigned long long* m_next,
               uint32_t* flags, uint32_t n, int half_bits, unsigned* ticket, unsigned* err,
               const Launch& L) {
  if (table == nullptr || slots == 0 || (slots & (slots - 1)) != 0 || slots > table_slots)
    return false;
  const uint32_t per_launch = (uint32_t)std::min<uint64_t>(kSegs, table_slots / slots);
  {
    KScope ks(L, kKSegDedup);
    k_seg_tiles<<<1, kSortThreads, 0, L.stream>>>(scratch);
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_insert, kSortThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const uint64_t max_tiles = (max_count + kSegInsTile - 1) / kSegInsTile + kSegs;
  const int grid = (int)std::min<uint64_t>(max_tiles, (uint64_t)L.sms * per_sm);
  for (uint32_t lo = 0; lo < kSegs; lo += per_launch) {
    const uint32_t hi = std::min(kSegs, lo + per_launch);
    cudaMemsetAsync(table, 0xFF, 8ull * slots * (hi - lo), L.stream);
    cudaMemsetAsync(ticket, 0, sizeof(unsigned), L.stream);
    KScope ks(L, kKSegDedup);
    k_seg_insert<<<grid, kSortThreads, 0, L.stream>>>(
        keys, scratch, lo, hi, slots, reinterpret_cast<unsigned long long*>(table), out,
        max_count, m_next, flags, n, half_bits, ticket, err);
  }
  return true;
}

void seg_compact(const uint64_t* keys, const uint32_t* scratch, uint64_t* out, const Launch& L) {
  KScope ks(L, kKSegDedup);
  k_seg_compact<<<kSegs, kSortThreads, 0, L.stream>>>(keys, scratch, out);
}

uint64_t sort_status_words(uint64_t max_keys) {
  uint64_t tiles = (max_keys + kSortTile - 1) / kSortTile;
  uint64_t w = tiles * kRadixMax;
  return std::max<uint64_t>(w, 1024);
}

uint32_t next_epoch(SortScratch& s, const Launch& L) {
  if (s.epoch == 0 || s.epoch >= (1u << 30) - 1) {
    cudaMemsetAsync(s.status, 0, s.status_words * sizeof(uint64_t), L.stream);
    s.epoch = 0;
  }
  return ++s.epoch;
}

static size_t sort_pass_smem(int rb) {
  return (size_t)kSortTile * 8 + (size_t)kWarps * (1u << rb) * 4 + (size_t)(1u << rb) * 4;
}

static size_t dedup_smem() { return (size_t)kTableSlots * (8 + 2); }

// Opt in to more than 48 KB of dynamic shared memory (a cheap host call,
// repeated before each use so every device the library runs on sees it).
static void set_smem_limits() {
  cudaFuncSetAttribute(k_sort_pass<kRadixBitsMax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sort_pass_smem(kRadixBitsMax));
  cudaFuncSetAttribute(k_bucket_dedup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)dedup_smem());
}

void hist_reset(SortScratch& s, const Launch& L) {
  cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * kMaxPasses * kRadixMax, L.stream);
}

// hist_ready: s.hist already holds the plan's digit counts (accumulated by the
// producer of the keys); otherwise a histogram pass reads the keys first.
static int run_passes(uint64_t* keys, uint64_t* alt, const unsigned long long* d_count,
                      uint64_t max_count, const PassPlan& plan, bool hist_ready, SortScratch& s,
                      unsigned* err, uint32_t* mark_flags, int half_bits, const Launch& L) {
  if (max_count == 0 || plan.passes == 0) return 0;
  set_smem_limits();
  cudaMemsetAsync(s.tickets, 0, sizeof(unsigned) * 8, L.stream);
  uint64_t tiles = (max_count + kSortTile - 1) / kSortTile;
  if (!hist_ready) {
    hist_reset(s, L);
    int hgrid = (int)std::min<uint64_t>(tiles, (uint64_t)L.sms * 4);
    KScope ks(L, kKSortHist);
    k_sort_hist<<<hgrid, kSortThreads, 0, L.stream>>>(keys, d_count, plan, s.hist);
  }
  {
    KScope ks(L, kKHistScan);
    k_hist_scan<<<plan.passes, kSortThreads, 0, L.stream>>>(s.hist);
  }
  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int p = 0; p < plan.passes; ++p) {
    uint32_t epoch = next_epoch(s, L);
    bool last = p == plan.passes - 1;
    KScope ks(L, kKSortPass);
    k_sort_pass<kRadixBitsMax><<<(unsigned)tiles, kSortThreads, sort_pass_smem(kRadixBitsMax),
                                 L.stream>>>(
        src, dst, d_count, plan.digit_fn(p), plan.bits[p], s.hist + p * kRadixMax, s.status,
        epoch, s.tickets + p, err, last ? mark_flags : nullptr, half_bits, s.spin_limit,
        p == 0 ? s.stall_once : 0);
    s.stall_once = 0;
    std::swap(src, dst);
  }
  return plan.passes & 1;
}

int radix_sort_u64(uint64_t* keys, uint64_t* alt, const unsigned long long* d_count,
                   uint64_t max_count, int key_bits, SortScratch& s, unsigned* err,
                   uint32_t* mark_flags, int half_bits, const Launch& L) {
  PassPlan plan{};
  plan.passes = (std::max(key_bits, 1) + kRadixBits - 1) / kRadixBits;
  for (int p = 0; p < plan.passes; ++p) {
    plan.shift[p] = kRadixBits * p;
    plan.bits[p] = kRadixBits;
  }
  return run_passes(keys, alt, d_count, max_count, plan, false, s, err, mark_flags, half_bits, L);
}

void filter_hll(const uint64_t* in, const unsigned long long* d_in, uint64_t max_count,
                uint64_t* out, unsigned long long* d_out, unsigned long long* gcache,
                uint32_t gslots, int admit, uint32_t* hll, const Launch& L) {
  if (max_count == 0) return;
  const int grid = (int)std::min<uint64_t>((max_count + kSortTile - 1) / kSortTile,
                                           (uint64_t)L.sms * 8);
  KScope ks(L, kKFilter);
  k_filter_hll<<<grid, kSortThreads, 0, L.stream>>>(in, d_in, out, d_out,
                                                    gslots ? gcache : nullptr,
                                                    gslots ? gslots - 1 : 0u, admit, hll);
}

int hash_bits_for(uint64_t max_count) {
  int b = 0;
  while (b < kMaxHashBits && ((uint64_t)kBucketTarget << b) < max_count) ++b;
  return b;
}

int hash_plan(uint64_t max_count, PassPlan* plan) {
  const int hb = hash_bits_for(max_count);
  *plan = PassPlan{};
  plan->passes = (hb + kRadixBitsMax - 1) / kRadixBitsMax;
  int shift = 64 - hb;  // the bucket is the top hb bits of the mixed key
  for (int p = 0; p < plan->passes; ++p) {
    int w = hb / plan->passes + (p < hb % plan->passes ? 1 : 0);
    plan->shift[p] = shift;
    plan->bits[p] = w;
    shift += w;
  }
  return hb;
}

int hash_dedup(uint64_t* keys, uint64_t* alt, const unsigned long long* d_count,
               uint64_t max_count, const PassPlan& plan, int hb, bool hist_ready,
               int half_bits, uint32_t* flags, uint32_t n, uint32_t* bounds,
               unsigned long long* m_next, SortScratch& s, unsigned* err, const Launch& L) {
  if (max_count == 0) return 0;
  int which =
      run_passes(keys, alt, d_count, max_count, plan, hist_ready, s, err, nullptr, half_bits, L);
  uint64_t* part = which ? alt : keys;
  uint64_t* out = which ? keys : alt;
  const uint32_t nb = 1u << hb;
  {
    KScope ks(L, kKBucketBounds);
    int g = (int)std::min<uint64_t>(((uint64_t)nb + 256) / 256, (uint64_t)L.sms * 8);
    k_bucket_bounds<<<g, 256, 0, L.stream>>>(part, d_count, hb, nb, bounds);
  }
  cudaMemsetAsync(s.tickets + 10, 0, sizeof(unsigned), L.stream);
  {
    KScope ks(L, kKBucketDedup);
    set_smem_limits();
    int g = (int)std::min<uint64_t>(nb, (uint64_t)L.sms * 6);
    k_bucket_dedup<<<g, kSortThreads, dedup_smem(), L.stream>>>(
        part, bounds, nb, out, max_count, m_next, flags, n, half_bits, s.tickets + 10, err);
  }
  return which;  // keys partitioned in `part` (0: keys, 1: alt); distinct keys in the other
}

void unmix_keys(uint64_t* e, const unsigned long long* d_count, uint64_t max_count,
                const Launch& L) {
  if (max_count == 0) return;
  KScope ks(L, kKUnmix);
  int g = (int)std::min<uint64_t>((max_count + 255) / 256, (uint64_t)L.sms * 8);
  k_unmix<<<g, 256, 0, L.stream>>>(e, d_count);
}

void rename_edges(uint64_t* e, const unsigned long long* d_count, uint64_t max_count,
                  int half_bits, const uint64_t* rank, uint32_t n, unsigned* err,
                  const Launch& L) {
  if (max_count == 0) return;
  KScope ks(L, kKRename);
  int g = (int)std::min<uint64_t>((max_count + 255) / 256, (uint64_t)L.sms * 8);
  k_rename<<<g, 256, 0, L.stream>>>(e, d_count, max_count, half_bits, rank, n, err);
}

void scan_flags(const uint32_t* flags, uint64_t* rank, uint32_t n, const uint32_t* mo_in,
                uint32_t* mo_out, unsigned long long* total, SortScratch& s, unsigned* err,
                const Launch& L) {
  if (n == 0) return;
  uint32_t epoch = next_epoch(s, L);
  cudaMemsetAsync(s.tickets + 8, 0, sizeof(unsigned), L.stream);
  uint64_t tiles = (rank_words(n) + kRankTile - 1) / kRankTile;
  KScope ks(L, kKScanFlags);
  k_scan_flags<<<(unsigned)tiles, kSortThreads, 0, L.stream>>>(flags, rank, n, mo_in, mo_out,
                                                              total, s.status, epoch,
                                                              s.tickets + 8, err);
}

void unique_rename(const uint64_t* keys, const unsigned long long* d_count, uint64_t max_count,
                   int half_bits, const uint64_t* rank, uint32_t n, uint64_t* out,
                   unsigned long long* m_next, SortScratch& s, unsigned* err, const Launch& L) {
  if (max_count == 0) return;
  uint32_t epoch = next_epoch(s, L);
  cudaMemsetAsync(s.tickets + 9, 0, sizeof(unsigned), L.stream);
  uint64_t tiles = (max_count + kScanTile - 1) / kScanTile;
  KScope ks(L, kKUniqueRename);
  k_unique_rename<<<(unsigned)tiles, kSortThreads, 0, L.stream>>>(
      keys, d_count, half_bits, rank, n, out, m_next, s.status, epoch, s.tickets + 9, err);
}

}  // namespace lc
