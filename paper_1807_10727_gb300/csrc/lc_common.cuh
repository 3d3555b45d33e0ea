// Device-side building blocks shared by the LocalContraction kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lc.h"

namespace lc {

// ---------------------------------------------------------------- ranking
// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): state advances by the golden-ratio increment and
// each output is the state passed through the variant-13 mixing function.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Phase key of vertex v: rank in the high 32 bits, id in the low 32 bits, so
// comparisons give a total order with ties broken by the smaller id.  `rk` is
// the phase's stream seed (output i+1 of the stream seeded with the run seed).
__device__ __forceinline__ uint64_t phase_key(uint64_t rk, uint32_t v) {
  return (splitmix_mix(rk + (uint64_t)(v + 1ull) * kGamma) & 0xFFFFFFFF00000000ull) | v;
}

// ---------------------------------------------------------------- errors
// Device error word bits (OR-ed in by kernels, read back by the host).
enum : uint32_t {
  kErrBadVertex = 1u,  // an input endpoint was >= n
  kErrTimeout = 2u,    // a bounded spin-wait gave up
  kErrOverflow = 4u,   // a dedup bucket held more distinct keys than its table
  kErrCorrupt = 8u,    // a data-dependent index was out of range (access skipped)
};

// Bijective mixer of an edge key (xorshift-multiply rounds).  The hashed
// dedup stores keys in mixed form: equal keys stay equal, the top bits pick
// the bucket and the low bits the hash-set slot, and key_unmix restores the
// key.  Any well-mixing bijection serves; the mixed form never reaches the
// output.
constexpr uint64_t kMixMul = 0xD6E8FEB86659FD93ull;
constexpr uint64_t kMixMulInv = 0xCFEE444D8B59A89Bull;  // kMixMul^-1 mod 2^64
static_assert(kMixMul * kMixMulInv == 1ull, "mix inverse");

__host__ __device__ __forceinline__ constexpr uint64_t key_mix(uint64_t k) {
  k ^= k >> 32;
  k *= kMixMul;
  k ^= k >> 32;
  k *= kMixMul;
  k ^= k >> 32;
  return k;
}

// x ^= x >> 32 is its own inverse; the multiplications undo with kMixMulInv.
__host__ __device__ __forceinline__ constexpr uint64_t key_unmix(uint64_t y) {
  y ^= y >> 32;
  y *= kMixMulInv;
  y ^= y >> 32;
  y *= kMixMulInv;
  y ^= y >> 32;
  return y;
}

// ~0 marks an empty hash-set slot.  It is never a mixed key: its preimage
// has a high half above its low half (not a < b for 32-bit halves) and is
// >= 2^62 (too wide for narrower halves).
static_assert((key_unmix(~0ull) >> 32) > (key_unmix(~0ull) & 0xFFFFFFFFull) &&
                  key_unmix(~0ull) >= (1ull << 62),
              "empty-slot sentinel collides with a key");

// Bucket of a mixed key: its top hb bits (0 when hb == 0).
__device__ __forceinline__ uint64_t bucket_of(uint64_t y, int hb) {
  return hb ? y >> (64 - hb) : 0ull;
}

// Iteration limit of every spin-wait on another block's status word.
constexpr uint32_t kSpinLimit = 1u << 24;

// Per-run device counters, read back once per phase with one small copy.
struct Counters {
  unsigned long long mprime;   // non-loop edges after relabelling (m'_i)
  unsigned long long m_next;   // distinct edges (m_{i+1})
  unsigned long long n_next;   // surviving nodes (n_{i+1})
  unsigned long long emitted;  // keys written by relabel (m'_i minus repeats it dropped)
  unsigned int err;            // kErr* bits
  unsigned int bad_kernel;     // 1 + kernel id of the first failed index check
  unsigned long long bad_index;
  unsigned long long bad_limit;
  unsigned long long tag;      // stamped by the last kernel of a phase (see run_complete)
  unsigned long long filtered; // keys left by the device-wide duplicate filter
};
static_assert(offsetof(Counters, bad_kernel) == offsetof(Counters, err) + 4, "layout");
static_assert(offsetof(Counters, bad_index) == offsetof(Counters, err) + 8, "layout");
static_assert(offsetof(Counters, bad_limit) == offsetof(Counters, err) + 16, "layout");

// atomicMin / atomicMax preceded by a read through L2: the stored values
// only move one way, so a read value is never past the current one, and a
// candidate that does not beat it cannot change the word.  Addresses that many
// threads update (hubs) then take few atomics instead of one per update.
__device__ __forceinline__ void min_if_lower(unsigned long long* p, unsigned long long v) {
  if (v < __ldcg(p)) atomicMin(p, v);
}
__device__ __forceinline__ void min_if_lower(unsigned* p, unsigned v) {
  if (v < __ldcg(p)) atomicMin(p, v);
}
__device__ __forceinline__ void max_if_higher(unsigned long long* p, unsigned long long v) {
  if (v > __ldcg(p)) atomicMax(p, v);
}

// Index check of a data-dependent access: false (and the first failure
// recorded next to the error word, see Counters) when idx >= limit.  Kernels
// skip the access when it fails, so corrupted data gives an error status, not
// a memory fault.
__device__ __forceinline__ bool index_ok(unsigned* err, uint32_t kernel, uint64_t idx,
                                         uint64_t limit) {
  if (idx < limit) return true;
  atomicOr(err, kErrCorrupt);
  if (atomicCAS(err + 1, 0u, kernel + 1) == 0u) {
    reinterpret_cast<unsigned long long*>(err + 2)[0] = idx;
    reinterpret_cast<unsigned long long*>(err + 2)[1] = limit;
  }
  return false;
}

// Node flags ("keeps an edge") are a bitmap: bit v & 31 of word v >> 5.  At
// one bit per node the array of a 2^26-node phase is 8 MB and stays in L2
// while the random marks land on it; byte flags (64 MB) did not.  A mark
// reads the word first: skewed graphs mark their hubs once per edge, and
// atomics on one address serialise, while a read of a set bit is a cache
// hit.  A stale read (another block set the bit since) only costs the atomic.
__host__ __device__ __forceinline__ constexpr uint64_t flag_words(uint64_t n) {
  return (n + 31) >> 5;
}
__device__ __forceinline__ void mark_flag(uint32_t* flags, uint64_t v) {
  uint32_t* w = flags + (v >> 5);
  const uint32_t bit = 1u << (v & 31);
  if ((*w & bit) == 0u) atomicOr(w, bit);
}

// Keep ranks of a level's nodes (a node is kept when it still has an edge
// after the relabel): word w of the rank_words(n) words holds, in its high
// half, the number of kept nodes below node 32w and, in its low half, the
// keep bits of nodes 32w..32w+31 (the last word covers node n, so the rank
// of n is the kept total).  A kept node's new id is one 8-byte read and a
// popcount, from 1/16 of the bytes of a per-node prefix: 16 MB at n = 2^26,
// which the renumbering's random reads find in L2.
__host__ __device__ __forceinline__ constexpr uint64_t rank_words(uint64_t n) {
  return (n >> 5) + 1;
}
// *id = number of kept nodes below v; returns whether v is kept (v <= n).
__device__ __forceinline__ bool keep_rank(const uint64_t* rank, uint32_t v, uint32_t* id) {
  const uint64_t x = __ldg(rank + (v >> 5));
  const uint32_t bits = (uint32_t)x, b = v & 31u;
  *id = (uint32_t)(x >> 32) + __popc(bits & ((1u << b) - 1u));
  return (bits >> b) & 1u;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// 64-bit status words of the single-pass (decoupled look-back) scans:
// [63:34] epoch, [33:32] flag, [31:0] value.
constexpr uint64_t kFlagAgg = 1ull;
constexpr uint64_t kFlagPrefix = 2ull;

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint64_t flag, uint32_t v) {
  return ((uint64_t)epoch << 34) | (flag << 32) | v;
}

__device__ __forceinline__ void store_status(uint64_t* p, uint64_t w) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ uint64_t load_status(const uint64_t* p) {
  uint64_t w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}

}  // namespace lc
