// Device helpers shared by the lookup kernels (lookup.cu, multi_lookup.cu): 128-bit compares, the
// branchless lower bound, and the search of the shared-memory top-of-tree index.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace planb {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kRounds = 4;  // addresses per 8-lane group in flight during the L2 levels

// 128-bit unsigned k < x
__device__ __forceinline__ bool less128(uint64_t kh, uint64_t kl, uint64_t xh, uint64_t xl) {
  return (kh < xh) | ((kh == xh) & (kl < xl));
}

#ifdef PLANB_BOUNDS_CHECK
__device__ __forceinline__ void report(uint32_t* status, uint32_t code) {
  if (status) atomicOr(status, code);
}
#endif

// Copies the high halves of index entries [0, n) (16-byte (high, low) entries in global memory)
// and the radix directory (dn u16 words) into shared memory, each thread with eight loads in
// flight, so an index of a few hundred KB arrives in a few L2 round trips rather than one per
// 8 bytes a thread copies. Ends with a barrier.
__device__ __forceinline__ void stage_index(uint64_t* Uh, const ulonglong2* sidx, uint32_t n,
                                            uint16_t* Dir, const uint16_t* dir, uint32_t dn) {
  constexpr uint32_t U = 8;
  for (uint32_t i0 = threadIdx.x; i0 < n; i0 += U * blockDim.x) {
    uint64_t v[U];
#pragma unroll
    for (uint32_t k = 0; k < U; k++) {
      const uint32_t i = i0 + k * blockDim.x;
      v[k] = i < n ? __ldg(&sidx[i].x) : 0ull;
    }
#pragma unroll
    for (uint32_t k = 0; k < U; k++) {
      const uint32_t i = i0 + k * blockDim.x;
      if (i < n) Uh[i] = v[k];
    }
  }
  for (uint32_t i0 = threadIdx.x; i0 < dn; i0 += U * blockDim.x) {
    uint16_t v[U];
#pragma unroll
    for (uint32_t k = 0; k < U; k++) {
      const uint32_t i = i0 + k * blockDim.x;
      v[k] = i < dn ? __ldg(dir + i) : uint16_t(0);
    }
#pragma unroll
    for (uint32_t k = 0; k < U; k++) {
      const uint32_t i = i0 + k * blockDim.x;
      if (i < dn) Dir[i] = v[k];
    }
  }
  __syncthreads();
}

// Number of entries of the sorted array a[0..n) that are below x (n >= 1), branch-free with a
// trip count that depends on n only (Khuong and Morin's branchless binary search).
template <class Load>
__device__ __forceinline__ uint32_t count_below(Load load, uint32_t n, uint64_t xh, uint64_t xl) {
  uint32_t b = 0;
  while (n > 1) {
    const uint32_t half = n >> 1;
    const ulonglong2 u = load(b + half);
    b = less128(u.x, u.y, xh, xl) ? b + half : b;
    n -= half;
  }
  const ulonglong2 u = load(b);
  return b + (less128(u.x, u.y, xh, xl) ? 1u : 0u);
}

// Entries of the staged index Uh[0..N) (ascending high halves) below the address, counting an
// entry with an equal high half by its low half (read from the global index). With a radix
// directory the search starts in the entries of the address's bucket: entries of lower buckets
// have smaller high halves, entries of higher buckets larger ones.
// An address's low half, read from memory the first time a comparison needs it (only when a key's
// high half equals the address's, which is rare), so the common lookup reads 8 bytes of address.
// (The address of the low half is passed to each get() rather than kept, to spare registers.)
// Where an address's low half lives: entry j of lo, or — for a multi-table launch over bucketed
// addresses — entry src[j] of the batch's input-order low halves, the bucketing having recorded
// each bucketed slot's input position instead of copying its low half. Only ptr() touches src.
struct LoRef {
  const uint64_t* lo;
  const uint32_t* src;
  uint64_t j;
  __device__ __forceinline__ const uint64_t* ptr() const { return lo + (src ? src[j] : j); }
};

struct LazyLo {
  uint64_t v;
  bool have;
  __device__ __forceinline__ explicit LazyLo(bool ok) : v(0), have(!ok) {}
  __device__ __forceinline__ uint64_t get(const LoRef& r) {
    if (!have) {
      v = *r.ptr();
      have = true;
    }
    return v;
  }
};

// The same count searched in place in global memory (the index's high halves at stride 16 bytes,
// the directory as stored), for launches too small to repay staging the index per CTA.
__device__ __forceinline__ uint32_t index_count_global(const ulonglong2* sidx, uint32_t N,
                                                       const uint16_t* dir, uint32_t dir_bits,
                                                       uint32_t dir_shift, uint64_t dir_base,
                                                       uint64_t my_hi, LazyLo& my_lo,
                                                       const LoRef& lo_src) {
  uint32_t lo = 0, n = N;
  if (dir_bits) {
    const uint64_t v = my_hi >> dir_shift;
    uint64_t bk = v > dir_base ? v - dir_base : 0ull;
    const uint64_t last = (1ull << dir_bits) - 1ull;
    bk = bk < last ? bk : last;
    lo = __ldg(dir + bk);
    n = __ldg(dir + bk + 1) - lo;
  }
  uint32_t cnt = lo;
  if (n) {
    uint32_t b = lo;
    while (n > 1) {
      const uint32_t half = n >> 1;
      b = __ldg(&sidx[b + half].x) < my_hi ? b + half : b;
      n -= half;
    }
    cnt = b + (__ldg(&sidx[b].x) < my_hi ? 1u : 0u);
  }
  while (cnt < N && __ldg(&sidx[cnt].x) == my_hi && __ldg(&sidx[cnt].y) < my_lo.get(lo_src)) cnt++;
  return cnt;
}

// Entries of the ascending array a[lo, lo + n) below x, searched branch-free over the n + 1
// possible answers lo .. lo + n: each read halves the candidates, ceil(log2(n + 1)) reads in all
// (against ceil(log2 n) + 1 for a search of the n entries that compares the last one it keeps).
template <class Load>
__device__ __forceinline__ uint32_t count_hi_below(Load a, uint32_t lo, uint32_t n, uint64_t x) {
  uint32_t b = lo, m = n + 1u;
  while (m > 1u) {
    const uint32_t half = m >> 1;
    b = a(b + half - 1u) < x ? b + half : b;
    m -= half;
  }
  return b;
}

// Entries of the staged high halves Uh[0..N) below the address's high half, started in the
// address's bucket of the radix directory (the high-half-only count of the F16HI descent).
__device__ __forceinline__ uint32_t index_count_hi(const uint64_t* Uh, uint32_t N,
                                                   const uint16_t* Dir, uint32_t dir_bits,
                                                   uint32_t dir_shift, uint64_t dir_base,
                                                   uint64_t my_hi) {
  uint32_t lo = 0, n = N;
  if (dir_bits) {
    const uint64_t v = my_hi >> dir_shift;
    uint64_t bk = v > dir_base ? v - dir_base : 0ull;
    const uint64_t last = (1ull << dir_bits) - 1ull;
    bk = bk < last ? bk : last;
    lo = Dir[bk];
    n = Dir[bk + 1] - lo;
  }
  return count_hi_below([Uh](uint32_t i) { return Uh[i]; }, lo, n, my_hi);
}

// The same count read in place from the global index (entries of 16 bytes, high half first) and
// directory, for launches too small to repay staging.
__device__ __forceinline__ uint32_t index_count_hi_global(const ulonglong2* sidx, uint32_t N,
                                                          const uint16_t* dir, uint32_t dir_bits,
                                                          uint32_t dir_shift, uint64_t dir_base,
                                                          uint64_t my_hi) {
  uint32_t lo = 0, n = N;
  if (dir_bits) {
    const uint64_t v = my_hi >> dir_shift;
    uint64_t bk = v > dir_base ? v - dir_base : 0ull;
    const uint64_t last = (1ull << dir_bits) - 1ull;
    bk = bk < last ? bk : last;
    lo = __ldg(dir + bk);
    n = __ldg(dir + bk + 1) - lo;
  }
  return count_hi_below([sidx](uint32_t i) { return __ldg(&sidx[i].x); }, lo, n, my_hi);
}

// Four consecutive high halves of a 128-byte F16HI node line (32 bytes, 32-byte aligned), read
// with one 256-bit load through the read-only path.
struct Quad {
  uint64_t a, b, c, d;
};
__device__ __forceinline__ Quad ldg_quad(const uint64_t* p) {
  Quad q;
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(q.a), "=l"(q.b), "=l"(q.c), "=l"(q.d)
      : "l"(p));
  return q;
}

// L2 eviction policies (sm_80+ createpolicy): evict-first for data streamed through once (a
// batch's addresses and results), evict-last for table lines that later lookups read again, so a
// large batch does not push a table set of L2's size out of it. (volatile: made where it is used,
// one instruction, rather than held in two registers across a loop)
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t ldg_hint_u64(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ldg_hint_u8(const uint8_t* p, uint64_t pol) {
  uint16_t v;
  asm("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ldg_hint_u32(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void stg_hint_u16(uint16_t* p, uint16_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(p), "h"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ Quad ldg_quad_hint(const uint64_t* p, uint64_t pol) {
  Quad q;
  asm("ld.global.nc.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
      : "=l"(q.a), "=l"(q.b), "=l"(q.c), "=l"(q.d)
      : "l"(p), "l"(pol));
  return q;
}

// Keys of a 16-key node below q for a 4-lane group (lane j of the group holds keys 4j .. 4j+3 in
// k): one ballot per key slot; bit 4g + j of ballot s is key 4j + s of group g, so the group's
// nibble of each of the four ballots, gathered into one word by byte permutes (`sel` picks byte
// g / 2 of two ballots, `nib` keeps the group's nibble of each byte), holds one bit per key below.
__device__ __forceinline__ uint32_t quad_count(const Quad& k, uint64_t q, uint32_t sel,
                                               uint32_t nib) {
  const uint32_t b0 = __ballot_sync(kFull, k.a < q);
  const uint32_t b1 = __ballot_sync(kFull, k.b < q);
  const uint32_t b2 = __ballot_sync(kFull, k.c < q);
  const uint32_t b3 = __ballot_sync(kFull, k.d < q);
  const uint32_t x = __byte_perm(__byte_perm(b0, b1, sel), __byte_perm(b2, b3, sel), 0x5410u);
  return __popc(x & nib);
}

// The same count searched in place with the bucket directory (see BucketDir): one 16-byte read
// of the address's bucket — its first entry's position, its entry count and that entry's high
// half — settles a bucket of at most one entry; a fuller one is finished by a branch-free search
// of its other entries in the global index. Buckets clamp at both ends: the entries of the first
// and last buckets are compared with the address like any other.
__device__ __forceinline__ uint32_t index_count_hi_bucket(const ulonglong2* sidx,
                                                          const ulonglong2* bdir, uint32_t bits,
                                                          uint32_t shift, uint64_t base,
                                                          uint64_t my_hi) {
  const uint64_t v = my_hi >> shift;
  uint64_t bk = v > base ? v - base : 0ull;
  const uint64_t last = (1ull << bits) - 1ull;
  bk = bk < last ? bk : last;
  const ulonglong2 w = __ldg(bdir + bk);
  const uint32_t start = static_cast<uint32_t>(w.x);
  const uint32_t n = static_cast<uint32_t>(w.x >> 32);
  if (n == 0u || w.y >= my_hi) return start;   // no entry of the bucket is below the address
  // the first is below: search the others
  return count_hi_below([sidx](uint32_t i) { return __ldg(&sidx[i].x); }, start + 1u, n - 1u,
                        my_hi);
}

// F16HI next-hop words: bits 0-15 the next hop of an interval, kTieBit set when the interval's key
// (its inclusive end) has a low half other than all-ones. Only such a key can be below an address
// whose high half it shares, so only there does a high-half-only count need a second look.
constexpr uint32_t kTieBit = 1u << 16;

// Settles a high-half-only count on the F16HI leaf level. `rank` counts the keys whose high half
// is below the address's; `w` is the next-hop word at that rank. Keys whose high half equals the
// address's follow in key order, sorted by low half, so the exact count adds the leading run of
// them whose low half is below the address's: found by doubling steps and then halving (a long
// run of /65+ boundaries inside one /64 costs a logarithmic number of reads). keys_hi / keys_lo
// are the leaf level's halves (key r at index r), nk the number of keys; lo() yields the address's
// low half. Returns the settled word and rank.
template <class Lo>
__device__ __forceinline__ uint32_t settle_tie(const uint64_t* keys_hi, const uint64_t* keys_lo,
                                               uint64_t nk, const uint32_t* words,
                                               uint64_t& rank, uint32_t w, uint64_t my_hi,
                                               Lo lo) {
  if (!(w & kTieBit) || __ldg(keys_hi + rank) != my_hi) return w;
  const uint64_t ql = lo();
  auto below = [&](uint64_t q) {
    return q < nk && __ldg(keys_hi + q) == my_hi && __ldg(keys_lo + q) < ql;
  };
  if (!below(rank)) return w;
  uint64_t good = rank, step = 1;
  while (below(rank + step)) {
    good = rank + step;
    step <<= 1;
  }
  uint64_t bad = rank + step;
  while (bad - good > 1) {
    const uint64_t mid = good + (bad - good) / 2;
    if (below(mid))
      good = mid;
    else
      bad = mid;
  }
  rank = bad;
  return __ldg(words + rank);
}

__device__ __forceinline__ uint32_t index_count(const uint64_t* Uh, uint32_t N,
                                                const uint16_t* Dir, uint32_t dir_bits,
                                                uint32_t dir_shift, uint64_t dir_base,
                                                const ulonglong2* sidx, uint64_t my_hi,
                                                LazyLo& my_lo, const LoRef& lo_src) {
  uint32_t lo = 0, n = N;
  if (dir_bits) {
    const uint64_t v = my_hi >> dir_shift;
    uint64_t bk = v > dir_base ? v - dir_base : 0ull;
    const uint64_t last = (1ull << dir_bits) - 1ull;
    bk = bk < last ? bk : last;
    lo = Dir[bk];
    n = Dir[bk + 1] - lo;
  }
  uint32_t cnt = lo;
  if (n) {
    uint32_t b = lo;
    while (n > 1) {
      const uint32_t half = n >> 1;
      b = Uh[b + half] < my_hi ? b + half : b;
      n -= half;
    }
    cnt = b + (Uh[b] < my_hi ? 1u : 0u);
  }
  while (cnt < N && Uh[cnt] == my_hi && __ldg(&sidx[cnt].y) < my_lo.get(lo_src)) cnt++;
  return cnt;
}

}  // namespace
}  // namespace planb
