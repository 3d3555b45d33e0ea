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

// Exclusive block scan of one value per thread (kSortThreads threads).
// `ws` must hold kWarps words; the call ends with a barrier so `ws` can be
// reused afterwards.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* ws,
                                                         uint32_t* total) {
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
// the exclusive prefix.  Every wait is bounded by kSpinLimit.
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
        --j;  // tile 0 always publishes a prefix, so j never wraps
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
                                                            int passes, uint32_t* ghist) {
  __shared__ uint32_t h[kMaxPasses][kRadix];
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint64_t count = *d_count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint64_t k = __ldcs(keys + i);
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (kRadixBits * p)) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// In-place exclusive scan of each pass's kRadix counts (one block per pass).
__global__ void __launch_bounds__(kRadix) k_hist_scan(uint32_t* ghist) {
  __shared__ uint32_t ws[kWarps];
  uint32_t* h = ghist + blockIdx.x * kRadix;
  uint32_t v = h[threadIdx.x], total;
  uint32_t e = block_exclusive_scan(v, ws, &total);
  h[threadIdx.x] = e;
}

// ------------------------------------------------------------ one pass

__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const uint64_t* __restrict__ in, uint64_t* __restrict__ out, const unsigned long long* d_count,
    int shift, const uint32_t* __restrict__ digit_offset, uint64_t* status, uint32_t epoch,
    unsigned* ticket, unsigned* err, uint8_t* mark_flags, int half_bits) {
  __shared__ uint64_t sk[kSortTile];
  __shared__ uint32_t whist[kWarps][kRadix];
  __shared__ uint32_t tstart[kRadix];
  __shared__ uint32_t gbase[kRadix];
  __shared__ uint32_t ws[kWarps];
  __shared__ uint32_t s_tile;
  __shared__ int s_bad;

  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(ticket, 1u);
    s_bad = 0;
  }
  for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t count = *d_count;
  const uint64_t base = (uint64_t)tile * kSortTile;
  if (base >= count) return;
  const uint32_t nvalid = (uint32_t)(count - base < (uint64_t)kSortTile ? count - base : (uint64_t)kSortTile);

  // load: warp w owns tile positions [w*32*kSortItems, (w+1)*32*kSortItems),
  // item i of lane l is position w*32*kSortItems + i*32 + l
  uint64_t k[kSortItems];
  uint32_t off[kSortItems];
  const uint32_t wbase = w * 32 * kSortItems;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    uint32_t pos = wbase + i * 32 + lane;
    k[i] = pos < nvalid ? __ldcs(in + base + pos) : ~0ull;
  }
  // stable warp-level ranking: earlier items, then lower lanes, come first
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    uint32_t pos = wbase + i * 32 + lane;
    uint32_t d = pos < nvalid ? (uint32_t)(k[i] >> shift) & (kRadix - 1) : (uint32_t)kRadix;
    unsigned peers = __match_any_sync(kFull, d);
    uint32_t r = __popc(peers & lanemask_lt());
    uint32_t cnt = d < (uint32_t)kRadix ? whist[w][d] : 0u;
    off[i] = cnt + r;
    __syncwarp();
    if (d < (uint32_t)kRadix && r == 0) whist[w][d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // per digit (one per thread): prefix over warps, tile count, look-back
  const uint32_t d = tid;
  uint32_t run = 0;
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) {
    uint32_t t = whist[ww][d];
    whist[ww][d] = run;
    run += t;
  }
  const uint32_t tcount = run;
  {
    // status words of this pass: [tile][digit] laid out digit-major per tile
    uint64_t* st = status + (uint64_t)tile * kRadix + d;
    uint32_t prefix = 0;
    if (tile == 0) {
      store_status(st, pack_status(epoch, kFlagPrefix, tcount));
    } else {
      store_status(st, pack_status(epoch, kFlagAgg, tcount));
      uint32_t j = tile - 1, spins = 0;
      for (;;) {
        uint64_t wd = load_status(status + (uint64_t)j * kRadix + d);
        if ((uint32_t)(wd >> 34) == epoch) {
          uint32_t flag = (uint32_t)(wd >> 32) & 3u;
          if (flag == kFlagPrefix) {
            prefix += (uint32_t)wd;
            break;
          }
          if (flag == kFlagAgg) {
            prefix += (uint32_t)wd;
            --j;
            spins = 0;
            continue;
          }
        }
        if (++spins > kSpinLimit) {
          atomicOr(err, kErrTimeout);
          s_bad = 1;
          break;
        }
      }
      store_status(st, pack_status(epoch, kFlagPrefix, prefix + tcount));
    }
    gbase[d] = digit_offset[d] + prefix;
  }
  uint32_t total;
  tstart[d] = block_exclusive_scan(tcount, ws, &total);
  __syncthreads();
  if (s_bad) return;  // offsets unknown: write nothing (the host sees kErrTimeout)

  // stage the tile in digit order
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    uint32_t pos = wbase + i * 32 + lane;
    if (pos < nvalid) {
      uint32_t dd = (uint32_t)(k[i] >> shift) & (kRadix - 1);
      sk[tstart[dd] + whist[w][dd] + off[i]] = k[i];
    }
  }
  __syncthreads();

  // coalesced write-out; optionally mark both endpoints of every key that
  // starts a run of equal keys inside the tile
  const uint64_t half_mask = (half_bits >= 64) ? ~0ull : ((1ull << half_bits) - 1);
  for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
    uint64_t key = sk[j];
    uint32_t dd = (uint32_t)(key >> shift) & (kRadix - 1);
    uint64_t gpos = (uint64_t)gbase[dd] + (j - tstart[dd]);
    if (gpos < count) out[gpos] = key;
    if (mark_flags != nullptr && (j == 0 || sk[j - 1] != key)) {
      mark_flags[key >> half_bits] = 1;
      mark_flags[key & half_mask] = 1;
    }
  }
}

// ------------------------------------------------------------- scans

constexpr int kScanItems = 16;
constexpr int kScanTile = kSortThreads * kScanItems;

__global__ void __launch_bounds__(kSortThreads) k_scan_flags(
    const uint8_t* __restrict__ flags, uint32_t* __restrict__ out, uint32_t n,
    const uint32_t* __restrict__ mo_in, uint32_t* __restrict__ mo_out,
    unsigned long long* total_out, uint64_t* status, uint32_t epoch, unsigned* ticket,
    unsigned* err) {
  __shared__ uint32_t ws[kWarps];
  __shared__ uint32_t s_tile, s_excl;
  const unsigned tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * kScanTile;
  if (base >= n) return;
  const uint64_t i0 = base + (uint64_t)tid * kScanItems;
  uint8_t f[kScanItems];
  if (i0 + kScanItems <= n) {
    uint4 q = *reinterpret_cast<const uint4*>(flags + i0);
    const uint8_t* b = reinterpret_cast<const uint8_t*>(&q);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) f[i] = b[i] ? 1 : 0;
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) f[i] = (i0 + i < n && flags[i0 + i]) ? 1 : 0;
  }
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) sum += f[i];
  uint32_t tile_total;
  uint32_t e = block_exclusive_scan(sum, ws, &tile_total);
  if (tid == 0) s_excl = look_back(status, tile, tile_total, epoch, err);
  __syncthreads();
  uint32_t run = s_excl + e;
  uint32_t o[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    o[i] = run;
    if (f[i] && mo_out != nullptr) mo_out[run] = mo_in[i0 + i];
    run += f[i];
  }
  if (i0 + kScanItems <= n) {
    uint4* dst = reinterpret_cast<uint4*>(out + i0);
#pragma unroll
    for (int i = 0; i < kScanItems / 4; ++i)
      dst[i] = make_uint4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
      if (i0 + i < n) out[i0 + i] = o[i];
  }
  if (base + kScanTile >= n && tid == 0) {
    uint32_t t = s_excl + tile_total;
    out[n] = t;
    *total_out = t;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_unique_rename(
    const uint64_t* __restrict__ keys, const unsigned long long* d_count, int half_bits,
    const uint32_t* __restrict__ newid, uint64_t* __restrict__ out, unsigned long long* m_next,
    uint64_t* status, uint32_t epoch, unsigned* ticket, unsigned* err) {
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
      uint32_t a = newid[k[i] >> half_bits];
      uint32_t b = newid[k[i] & half_mask];
      out[pos++] = ((uint64_t)a << 32) | b;
    }
  }
  if (base + kScanTile >= count && tid == 0) *m_next = (unsigned long long)s_excl + tile_total;
}

}  // namespace

// ------------------------------------------------------------- host side

uint64_t sort_status_words(uint64_t max_keys) {
  uint64_t tiles = (max_keys + kSortTile - 1) / kSortTile;
  uint64_t w = tiles * kRadix;
  return std::max<uint64_t>(w, 1024);
}

uint32_t next_epoch(SortScratch& s, const Launch& L) {
  if (s.epoch == 0 || s.epoch >= (1u << 30) - 1) {
    cudaMemsetAsync(s.status, 0, s.status_words * sizeof(uint64_t), L.stream);
    s.epoch = 0;
  }
  return ++s.epoch;
}

int radix_sort_u64(uint64_t* keys, uint64_t* alt, const unsigned long long* d_count,
                   uint64_t max_count, int key_bits, SortScratch& s, unsigned* err,
                   uint8_t* mark_flags, int half_bits, const Launch& L) {
  if (max_count == 0) return 0;
  int passes = (std::max(key_bits, 1) + kRadixBits - 1) / kRadixBits;
  cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * kMaxPasses * kRadix, L.stream);
  cudaMemsetAsync(s.tickets, 0, sizeof(unsigned) * 16, L.stream);
  uint64_t tiles = (max_count + kSortTile - 1) / kSortTile;
  int hgrid = (int)std::min<uint64_t>(tiles, (uint64_t)L.sms * 4);
  {
    KScope ks(L, kKSortHist);
    k_sort_hist<<<hgrid, kSortThreads, 0, L.stream>>>(keys, d_count, passes, s.hist);
  }
  {
    KScope ks(L, kKHistScan);
    k_hist_scan<<<passes, kRadix, 0, L.stream>>>(s.hist);
  }
  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int p = 0; p < passes; ++p) {
    uint32_t epoch = next_epoch(s, L);
    bool last = p == passes - 1;
    KScope ks(L, kKSortPass);
    k_sort_pass<<<(unsigned)tiles, kSortThreads, 0, L.stream>>>(
        src, dst, d_count, kRadixBits * p, s.hist + p * kRadix, s.status, epoch, s.tickets + p,
        err, last ? mark_flags : nullptr, half_bits);
    std::swap(src, dst);
  }
  return passes & 1;
}

void scan_flags(const uint8_t* flags, uint32_t* out, uint32_t n, const uint32_t* mo_in,
                uint32_t* mo_out, unsigned long long* total, SortScratch& s, unsigned* err,
                const Launch& L) {
  if (n == 0) return;
  uint32_t epoch = next_epoch(s, L);
  cudaMemsetAsync(s.tickets + 8, 0, sizeof(unsigned), L.stream);
  uint64_t tiles = ((uint64_t)n + kScanTile - 1) / kScanTile;
  KScope ks(L, kKScanFlags);
  k_scan_flags<<<(unsigned)tiles, kSortThreads, 0, L.stream>>>(flags, out, n, mo_in, mo_out, total,
                                                              s.status, epoch, s.tickets + 8, err);
}

void unique_rename(const uint64_t* keys, const unsigned long long* d_count, uint64_t max_count,
                   int half_bits, const uint32_t* newid, uint64_t* out,
                   unsigned long long* m_next, SortScratch& s, unsigned* err, const Launch& L) {
  if (max_count == 0) return;
  uint32_t epoch = next_epoch(s, L);
  cudaMemsetAsync(s.tickets + 9, 0, sizeof(unsigned), L.stream);
  uint64_t tiles = (max_count + kScanTile - 1) / kScanTile;
  KScope ks(L, kKUniqueRename);
  k_unique_rename<<<(unsigned)tiles, kSortThreads, 0, L.stream>>>(
      keys, d_count, half_bits, newid, out, m_next, s.status, epoch, s.tickets + 9, err);
}

}  // namespace lc
