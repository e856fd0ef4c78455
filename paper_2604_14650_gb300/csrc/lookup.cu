// Lookup kernels: descent of the linearized B+-tree for a batch of 128-bit addresses
// (hot-path steps a5-a10).
//
// The paper's search (Algorithm 1, Listing 1, Sections 3.2-3.5) runs one address per core through
// D node visits, each an 8-wide SIMD compare, a popcount and the child arithmetic
// i = (k+1) i + (c+1) k. On the GPU a node visit is spread over a lane group: lane j of an 8-lane
// group holds key j of the node (one 16-byte load; the group's 8 loads are one coalesced 128-byte
// line), compares it with the address as a 128-bit number, and the warp's ballot plus a popcount
// of the group's byte give every lane the child index c. The child of node i is node b*i + 1 + c
// (Section 3.2's child_start formula counted in nodes).
//
// Keys are the inclusive interval ends and every count is of keys strictly below the address, so
// the popcount at the leaf is the interval index r itself and the next hop is values[r] (the
// separate value array of Section 3.2).
//
// Node formats: F8X128 (8 keys per node, next hops in a separate array), F8V7 (internal nodes as
// F8X128; a leaf line holds 7 keys and their 7 next hops, so the descent's last load also brings
// the result), F16HI (16 high halves per node plus a low-half array).
//
// Three kernels:
//   coop    every level by 8-lane groups (16-lane groups for the F16HI format); the first
//           smem_levels levels are staged in shared memory per CTA. Four addresses per warp step.
//   hybrid  (default) levels 0 .. S-1 are replaced by a per-thread branchless lower bound over the
//           level-S subtree maxima staged in shared memory (the same count a descent of those
//           levels yields, at one 8-byte high half per level-S node instead of a 128-byte node per
//           internal node), started inside the address's bucket of a radix directory over those
//           high halves; the remaining D - S levels, read from L2, are descended by 8-lane
//           groups with four addresses per group in flight, so a warp keeps 16 node fetches
//           outstanding. The address-to-group broadcast of the paper's vector broadcast (Listing
//           1's set1) is a warp shuffle. On F16HI tables (16 high halves per line) the groups are
//           four lanes wide, each lane comparing four keys from one 32-byte load.
//   flat    per-thread lower bound over the whole sorted key array in global memory: the GPU
//           analogue of the paper's ablation baseline (Section 4.5, std::lower_bound).
// All are persistent: a grid of a few CTAs per SM strides over 32-address tiles; each lane owns
// one address of a tile, so address loads (8-byte hi and lo words) and next-hop stores (u16) are
// coalesced.
#include <cuda_runtime.h>

#include <algorithm>

#include "descent.cuh"
#include "learned.cuh"
#include "planb_internal.h"

namespace planb {

namespace {


struct KParams {
  const ulonglong2* nodes;    // F8X128 nodes (key j of node i at nodes[i*8 + j])
  const uint64_t* nodes_hi;   // F16HI high halves (key j of node i at [i*16 + j])
  const uint64_t* nodes_lo;   // F16HI low halves
  const ulonglong2* sidx;     // hybrid top-of-tree index
  const uint16_t* values;
  const uint32_t* nh_tie;     // F16HI: next-hop words (bits 0-15 next hop, kTieBit)
  const uint64_t* xhi;
  const uint64_t* xlo;
  uint16_t* out;
  uint64_t n;
  uint64_t n_intervals;
  uint64_t total_nodes;
  uint32_t internal_nodes;
  uint32_t smem_levels;
  uint32_t smem_nodes;
  uint32_t sidx_n;
  uint32_t sidx_node;
  uint32_t* status;
  const LeafModel* leaves;    // learned: leaf models (copied to shared memory)
  const uint16_t* leaf_err;   // learned: per-leaf window half-width or kLeafFallback
  LearnedParams lp;           // learned: root weights and range reduction
  uint32_t staged;            // hybrid: 1 = index and directory staged in shared memory, 0 =
                              // searched in place (small launches; no shared memory given)
  const uint16_t* dir;        // hybrid: radix directory over the index (dir_bits = 0: none)
  const ulonglong2* bdir;     // F16HI hybrid: bucket directory of the in-place search, or null
  BucketDir bdp;
  uint32_t dir_bits, dir_shift;
  uint64_t dir_base;
  const uint64_t* range;      // multi-table: device [begin, end) of this launch's addresses
  const uint32_t* src;        // multi-table: input position of bucketed address j; xlo is then
                              // the batch's input-order low halves, read at src[j] on a tie
};

// The addresses a launch handles: [0, n), or the device-side range a bucketing pass wrote.
struct Seg {
  uint64_t off, n;
};

template <bool MULTI = true>
__device__ __forceinline__ Seg segment(const KParams& p) {
  if (!MULTI || !p.range) return Seg{0, p.n};
  const uint64_t b = p.range[0], e = p.range[1];
  return Seg{b, e > b ? e - b : 0};
}

template <bool MULTI = true>
__device__ __forceinline__ void store_out(const KParams& p, uint64_t j, uint16_t v) {
  p.out[j] = v;
}

// The low half of address j of a launch (j counted from the start of the address arrays).
template <bool MULTI>
__device__ __forceinline__ LoRef lo_ref(const KParams& p, uint64_t j) {
  return LoRef{p.xlo, MULTI ? p.src : nullptr, j};
}

// ------------------------------------------------------------------------------- coop F8X128
template <int D>
__global__ void __launch_bounds__(256, 4) lookup_coop_f8(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* sm = reinterpret_cast<ulonglong2*>(smem_raw);
  const uint32_t staged = p.smem_nodes * 8u;
  for (uint32_t i = threadIdx.x; i < staged; i += blockDim.x) sm[i] = __ldg(p.nodes + i);
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t g = lane >> 3;        // group: which of the 4 addresses of a step
  const uint32_t j = lane & 7u;        // key slot in a node
  const uint32_t gshift = g * 8u;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint32_t S = p.smem_levels;

  const Seg seg = segment(p);
  for (uint64_t base = warp * 32; base < seg.n; base += nwarps * 32) {
    const uint64_t mine = base + lane;
    const bool ok = mine < seg.n;
    const uint64_t my_hi = ok ? p.xhi[seg.off + mine] : 0ull;
    const uint64_t my_lo = ok ? *lo_ref<true>(p, seg.off + mine).ptr() : 0ull;
    uint32_t result = 0;
#pragma unroll
    for (uint32_t r = 0; r < 8; r++) {
      // group g serves the address owned by its own lane r
      const uint64_t qh = __shfl_sync(kFull, my_hi, gshift + r);
      const uint64_t ql = __shfl_sync(kFull, my_lo, gshift + r);
      uint32_t node = 0, c = 0;
#pragma unroll
      for (int l = 0; l < D; l++) {
        ulonglong2 key;
        if (static_cast<uint32_t>(l) < S) key = sm[node * 8u + j];
        else key = __ldg(p.nodes + static_cast<uint64_t>(node) * 8u + j);
        const uint32_t m = __ballot_sync(kFull, less128(key.x, key.y, qh, ql));
        c = __popc((m >> gshift) & 0xFFu);
        if (l + 1 < D) node = node * 9u + 1u + c;
      }
      uint64_t rank = static_cast<uint64_t>(node - p.internal_nodes) * 8u + c;
#ifdef PLANB_BOUNDS_CHECK
      if (rank >= p.n_intervals || node >= p.total_nodes) {
        report(p.status, 1u);
        rank = 0;
      }
#endif
      const uint32_t v = __ldg(p.values + rank);
      if (j == r) result = v;
    }
    if (ok) store_out(p, seg.off + mine, static_cast<uint16_t>(result));
  }
}

// ------------------------------------------------------------------------------- coop F16HI
// 16-lane groups, two addresses per warp step; a node is 16 high halves (one 128-byte line). The
// descent counts high halves only (the count of keys whose high half is below the address's); the
// next-hop word at that count says whether a key sharing the address's high half could still be
// below it, and settle_tie finishes the count in that rare case.
template <int D>
__global__ void __launch_bounds__(256, 4) lookup_coop_f16(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem_raw);
  const uint32_t staged = p.smem_nodes * 16u;
  for (uint32_t i = threadIdx.x; i < staged; i += blockDim.x) sm[i] = __ldg(p.nodes_hi + i);
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t g = lane >> 4;
  const uint32_t j = lane & 15u;
  const uint32_t gshift = g * 16u;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint32_t S = p.smem_levels;
  const uint64_t leaf_key0 = static_cast<uint64_t>(p.internal_nodes) * 16u;
  const uint64_t nk = p.n_intervals - 1;

  const Seg seg = segment(p);
  for (uint64_t base = warp * 32; base < seg.n; base += nwarps * 32) {
    const uint64_t mine = base + lane;
    const bool ok = mine < seg.n;
    const uint64_t my_hi = ok ? p.xhi[seg.off + mine] : 0ull;
    const uint64_t my_lo = ok ? *lo_ref<true>(p, seg.off + mine).ptr() : 0ull;
    uint32_t result = 0;
#pragma unroll 4
    for (uint32_t r = 0; r < 16; r++) {
      const uint64_t qh = __shfl_sync(kFull, my_hi, gshift + r);
      const uint64_t ql = __shfl_sync(kFull, my_lo, gshift + r);
      uint32_t node = 0, c = 0;
#pragma unroll
      for (int l = 0; l < D; l++) {
        const uint64_t idx = static_cast<uint64_t>(node) * 16u + j;
        const uint64_t kh = (static_cast<uint32_t>(l) < S) ? sm[idx] : __ldg(p.nodes_hi + idx);
        const uint32_t m = __ballot_sync(kFull, kh < qh);
        c = __popc((m >> gshift) & 0xFFFFu);
        if (l + 1 < D) node = node * 17u + 1u + c;
      }
      uint64_t rank = static_cast<uint64_t>(node - p.internal_nodes) * 16u + c;
#ifdef PLANB_BOUNDS_CHECK
      if (rank >= p.n_intervals || node >= p.total_nodes) {
        report(p.status, 1u);
        rank = 0;
      }
#endif
      uint32_t w = __ldg(p.nh_tie + rank);
      w = settle_tie(p.nodes_hi + leaf_key0, p.nodes_lo + leaf_key0, nk, p.nh_tie, rank, w, qh,
                     [ql] { return ql; });
      if (j == r) result = w;
    }
    if (ok) store_out(p, seg.off + mine, static_cast<uint16_t>(result));
  }
}

// ------------------------------------------------------------------------------- hybrid
// DB = levels left after the shared-memory index (D - S); 0 when the index holds every key.
//
// Only the index's 8-byte high halves sit in shared memory (half the footprint and half the
// shared-memory wavefronts of 16-byte entries). The binary search counts the entries whose high
// half is below the address's; the entries whose high half equals it — contiguous and sorted by low
// half right after that count — are then added one by one while their low half, read from the
// global copy of the index, is below the address's (a /65+ boundary sharing the address's high
// half; rare, and a short loop when it happens).
//
// In the L2 levels a group needs the address of the lane it serves: only the high half and the node
// index are broadcast; the low half is broadcast only when some lane of the warp finds a key whose
// high half equals the address's.

//
// LEARNED: phase A first asks the learned position model (learned.cuh) for the address's interval
// rank and its leaf's recorded error e; the index entries that can hold the answer are those of the
// buckets of ranks [rank - e, rank + e], and a short search among them gives the count — accepted
// only when the entries just outside the window bracket the address (so the count is exact whatever
// the model said). Otherwise, and for leaves marked for the tree, the full binary search runs.
template <int DB, bool PACKED, bool LEARNED, bool MULTI, bool LAZY = false>
__global__ void __launch_bounds__(512, 2) lookup_hybrid(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t N = p.sidx_n;
  uint64_t* Uh = reinterpret_cast<uint64_t*>(smem_raw);
  // a small launch searches the index in place instead of staging it (decided by the host;
  // the learned and multi-table forms always stage)
  const bool staged = LEARNED || MULTI || p.staged != 0;
  uint16_t* Dir = reinterpret_cast<uint16_t*>(Uh + ((N + 1u) & ~1u));
  const uint32_t dn = p.dir_bits ? (1u << p.dir_bits) + 1u : 0u;
  if (staged && MULTI) {
    stage_index(Uh, p.sidx, N, Dir, p.dir, dn);
  } else if (staged) {
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) Uh[i] = __ldg(&p.sidx[i].x);
    for (uint32_t i = threadIdx.x; i < dn; i += blockDim.x) Dir[i] = __ldg(p.dir + i);
  }
  LeafModel* Lm = reinterpret_cast<LeafModel*>(Dir + ((dn + 7u) & ~7u));
  uint16_t* Le = reinterpret_cast<uint16_t*>(Lm + (LEARNED ? p.lp.leaves : 0u));
  if (LEARNED) {
    for (uint32_t i = threadIdx.x; i < p.lp.leaves; i += blockDim.x) {
      Lm[i] = p.leaves[i];
      Le[i] = p.leaf_err[i];
    }
  }
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  // 4-lane groups of phase B: group g, lane j within it; `sel` and `nib` gather the group's
  // nibble of two ballots into one word
  const uint32_t g = lane >> 2;
  const uint32_t j = lane & 3u;
  const uint32_t gmask = 0xFu << (g * 4u);
  const uint32_t sel = (g >> 1) | ((4u + (g >> 1)) << 4);
  const uint32_t nib = (g & 1u) ? 0xF0F0u : 0x0F0Fu;
  const uint64_t* nodes64 = reinterpret_cast<const uint64_t*>(p.nodes);
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;

  const Seg seg = segment<MULTI>(p);
  // the addresses of a warp's next tile are loaded while it works on the current one, so the
  // stream's HBM latency overlaps the descent
  // LAZY (addresses in host memory, read over the host link): an address's low half is read only
  // on a high-half tie; otherwise it is loaded, and prefetched, with the high half
  uint64_t nx_hi = 0, nx_lo = 0;
  {
    const uint64_t first = warp * 32 + lane;
    if (first < seg.n) {
      nx_hi = p.xhi[seg.off + first];
      if (!LAZY) nx_lo = p.xlo[seg.off + first];
    }
  }
  for (uint64_t base = warp * 32; base < seg.n; base += nwarps * 32) {
    const uint64_t mine = base + lane;
    const bool ok = mine < seg.n;
    const uint64_t my_hi = nx_hi;
    LazyLo my_lo(ok);
    if (!LAZY) {
      my_lo.v = nx_lo;
      my_lo.have = true;
    }
    const LoRef lo_src = lo_ref<MULTI>(p, seg.off + mine);
    {
      const uint64_t next = mine + nwarps * 32;
      nx_hi = next < seg.n ? p.xhi[seg.off + next] : 0ull;
      if (!LAZY) nx_lo = next < seg.n ? p.xlo[seg.off + next] : 0ull;
    }
    // phase A: per-thread count over the level-S subtree maxima in shared memory
    uint32_t cnt = 0;
    bool have = false;
    if constexpr (LEARNED) {
      auto below = [&](uint32_t q) {   // index entry q < address
        const uint64_t h = Uh[q];
        return h < my_hi || (h == my_hi && __ldg(&p.sidx[q].y) < my_lo.get(lo_src));
      };
      const uint32_t leaf = predict_leaf(p.lp, my_hi);
      const uint32_t e = Le[leaf];
      if (e != kLeafFallback) {
        const uint32_t r = predict_rank(p.lp, Lm[leaf], my_hi);
        const uint32_t lo_r = r > e ? r - e : 0u;
        const uint32_t hi_r = min(r + e, p.lp.n_keys - 1u);
        const uint32_t qa = min(div_span(p.lp, lo_r), N);
        const uint32_t qb = min(div_span(p.lp, hi_r), N);
        bool ok = qa == 0u || below(qa - 1u);
        ok = ok && (qb >= N || !below(qb));
        uint32_t b = qa, len = qb - qa;   // count the entries of [qa, qb) below the address
        while (len > 0u) {
          const uint32_t half = len >> 1;
          if (below(b + half)) {
            b += half + 1u;
            len -= half + 1u;
          } else {
            len = half;
          }
        }
        cnt = b;
        have = ok;
      }
    }
    if (N && !have && staged)
      cnt = index_count(Uh, N, Dir, p.dir_bits, p.dir_shift, p.dir_base, p.sidx, my_hi, my_lo,
                        lo_src);
    else if (N && !have)
      cnt = index_count_global(p.sidx, N, p.dir, p.dir_bits, p.dir_shift, p.dir_base, my_hi,
                               my_lo, lo_src);
    if constexpr (DB == 0) {
      uint32_t rank = cnt;
#ifdef PLANB_BOUNDS_CHECK
      if (rank >= p.n_intervals) {
        report(p.status, 2u);
        rank = 0;
      }
#endif
      const uint16_t v = __ldg(p.values + rank);
      if (ok) store_out<MULTI>(p, seg.off + mine, v);
    } else {
      const uint32_t my_node = p.sidx_node + cnt;
      uint32_t result = 0;
      uint64_t my_rank = 0;   // the interval index of this lane's own address
      // phase B: the last DB levels from L2 by 4-lane groups — lane j of group g holds keys 2j and
      // 2j + 1 of a node (one 32-byte load of two (high, low) pairs), the group's four addresses
      // are those of lanes 4g .. 4g + 3; one level left: all four in flight, else two at a time
      // (and two when the low half is read lazily: the registers it needs)
      constexpr int R = (DB == 1 && !LAZY) ? 4 : 2;
#pragma unroll
      for (int r0 = 0; r0 < 4; r0 += R) {
        uint64_t qh[R];
        uint32_t nd[R], c[R];
        Quad kq[R];
#pragma unroll
        for (int i = 0; i < R; i++) {
          const uint32_t src = g * 4u + r0 + i;
          qh[i] = __shfl_sync(kFull, my_hi, src);
          nd[i] = __shfl_sync(kFull, my_node, src);
        }
#pragma unroll
        for (int l = 0; l < DB; l++) {
#pragma unroll
          for (int i = 0; i < R; i++)
            kq[i] = ldg_quad(nodes64 + static_cast<uint64_t>(nd[i]) * 16u + j * 4u);
          const bool last = l + 1 == DB;
          // in a packed leaf, slot 7 (lane 3's second key) holds next hops, not a key
          const bool key1 = !PACKED || !last || j < 3u;
          // (few predicates live at once: the equalities are recomputed on the tie path)
          bool anyeq = false;
#pragma unroll
          for (int i = 0; i < R; i++)
            anyeq |= (kq[i].a == qh[i]) | (key1 & (kq[i].c == qh[i]));
          const bool tie = __any_sync(kFull, anyeq);
#pragma unroll
          for (int i = 0; i < R; i++) {
            bool lt0 = kq[i].a < qh[i];
            bool lt1 = key1 & (kq[i].c < qh[i]);
            if (tie) {
              const bool eq0 = kq[i].a == qh[i];
              const bool eq1 = key1 & (kq[i].c == qh[i]);
              // the owner of address i of each group reads its low half if its group saw a tie
              const uint32_t need = __ballot_sync(kFull, eq0 | eq1) & gmask;
              if (need && j == static_cast<uint32_t>(r0 + i)) my_lo.get(lo_src);
              const uint64_t ql = __shfl_sync(kFull, my_lo.v, g * 4u + r0 + i);
              lt0 = lt0 | (eq0 & (kq[i].b < ql));
              lt1 = lt1 | (eq1 & (kq[i].d < ql));
            }
            c[i] = __popc(__byte_perm(__ballot_sync(kFull, lt0), __ballot_sync(kFull, lt1), sel) &
                          nib);
            if (!last) nd[i] = nd[i] * 9u + 1u + c[i];
          }
          if (PACKED && last) {
            // the next hop of slot c sits in slot 7 of the same leaf line: lane 3 of the group
            // picks its 16-bit field and broadcasts it
#pragma unroll
            for (int i = 0; i < R; i++) {
#ifdef PLANB_BOUNDS_CHECK
              if (c[i] > 6u || nd[i] >= p.total_nodes) report(p.status, 4u);
#endif
              const uint32_t ci = c[i] & 7u;
              const uint64_t w = ci < 4u ? kq[i].c : kq[i].d;
              const uint32_t f = static_cast<uint32_t>(w >> (16u * (ci & 3u))) & 0xFFFFu;
              const uint32_t v = __shfl_sync(kFull, f, g * 4u + 3u);
              if (j == static_cast<uint32_t>(r0 + i)) result = v;
            }
          }
        }
        if (!PACKED) {
#pragma unroll
          for (int i = 0; i < R; i++) {
            uint64_t rank = static_cast<uint64_t>(nd[i] - p.internal_nodes) * 8u + c[i];
#ifdef PLANB_BOUNDS_CHECK
            if (rank >= p.n_intervals || nd[i] >= p.total_nodes) {
              report(p.status, 4u);
              rank = 0;
            }
#endif
            if (j == static_cast<uint32_t>(r0 + i)) my_rank = rank;
          }
        }
      }
      // each lane fetches its own next hop: one load per lane rather than one per group lane
      if (!PACKED) result = __ldg(p.values + my_rank);
      if (ok) store_out<MULTI>(p, seg.off + mine, static_cast<uint16_t>(result));
    }
  }
}

// ------------------------------------------------------------------------------- hybrid, F16HI
// The hybrid descent on the F16HI layout (17-ary nodes of 16 high halves, low halves in a parallel
// array). 16 keys per leaf make the leaf level small enough that the index over it fits one CTA's
// shared memory at backbone size, so phase B is often the leaf line alone: one dependent L2 round
// trip before the next hop instead of two. One 1024-thread CTA per SM holds the index; in phase B
// lane j of a 4-lane group loads the high halves of keys 4j .. 4j+3 with one 32-byte load (the
// group's four loads are the node's one 128-byte line), so one warp-wide load serves eight
// addresses, and the count is the population of the group's nibble of four ballots.
// Every level, the index included, counts high halves only; the next-hop word at the resulting
// count says whether a key sharing the address's high half could still be below the address, and
// settle_tie finishes the count then. An address's low half is read only in that case.
// MULTI: one table's launch within a multi-table batch (device-side address range, results through
// the permutation when one is given).
// IPB > 0: the in-place form's launch bounds, IPB 256-thread CTAs per SM (no shared memory).
template <int DB, bool MULTI = false, int IPB = 0>
__global__ void __launch_bounds__(IPB ? 256 : 1024, IPB ? IPB : 1) lookup_hybrid16(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t N = p.sidx_n;
  uint64_t* Uh = reinterpret_cast<uint64_t*>(smem_raw);
  uint16_t* Dir = reinterpret_cast<uint16_t*>(Uh + ((N + 1u) & ~1u));
  // a small launch searches the index in place instead of staging it (decided by the host)
  const bool staged = MULTI || p.staged != 0;
  if (staged) {
    const uint32_t dn = p.dir_bits ? (1u << p.dir_bits) + 1u : 0u;
    if (MULTI) {   // a table's share of a batch: staging is a larger part of the launch
      stage_index(Uh, p.sidx, N, Dir, p.dir, dn);
    } else {       // (the unrolled copy measured slower here: 75.2 against 79.1 B lookups/s)
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) Uh[i] = __ldg(&p.sidx[i].x);
      for (uint32_t i = threadIdx.x; i < dn; i += blockDim.x) Dir[i] = __ldg(p.dir + i);
      __syncthreads();
    }
  }

  const uint32_t lane = threadIdx.x & 31u;
  // phase B by 4-lane groups: lane j of group g holds keys 4j .. 4j+3 of a node (one 32-byte load),
  // so a warp works on eight nodes per load and each group has its four addresses in flight
  const uint32_t g = lane >> 2;
  const uint32_t j = lane & 3u;
  const uint32_t sel = (g >> 1) | ((4u + (g >> 1)) << 4);
  const uint32_t nib = (g & 1u) ? 0xF0F0F0F0u : 0x0F0F0F0Fu;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t leaf_key0 = static_cast<uint64_t>(p.internal_nodes) * 16u;
  const uint64_t nk = p.n_intervals - 1;

  const Seg seg = segment<MULTI>(p);
  const uint64_t* xhi = p.xhi + seg.off;
  uint64_t nx_hi = 0;
  {
    const uint64_t first = warp * 32 + lane;
    if (first < seg.n) nx_hi = xhi[first];
  }
  for (uint64_t base = warp * 32; base < seg.n; base += nwarps * 32) {
    const uint64_t mine = base + lane;
    const bool ok = mine < seg.n;
    const uint64_t my_hi = nx_hi;
    {
      const uint64_t next = mine + nwarps * 32;
      nx_hi = next < seg.n ? xhi[next] : 0ull;
    }
    uint32_t cnt = 0;
    if (N && staged)
      cnt = index_count_hi(Uh, N, Dir, p.dir_bits, p.dir_shift, p.dir_base, my_hi);
    else if (N && p.bdir)
      cnt = index_count_hi_bucket(p.sidx, p.bdir, p.bdp.bits, p.bdp.shift, p.bdp.base, my_hi);
    else if (N)
      cnt = index_count_hi_global(p.sidx, N, p.dir, p.dir_bits, p.dir_shift, p.dir_base, my_hi);
    uint64_t rank = cnt;
    if constexpr (DB > 0) {
      uint32_t my_node = p.sidx_node + cnt;
      uint32_t my_c = 0;
      // all four addresses of a group in flight when only the leaf level is left; deeper descents
      // carry node indexes across levels and take two at a time (register budget)
      constexpr int R = DB == 1 ? 4 : 2;
#pragma unroll
      for (int r0 = 0; r0 < 4; r0 += R) {
        uint64_t qh[R];
        uint32_t nd[R];
#pragma unroll
        for (int i = 0; i < R; i++) {
          const uint32_t src = g * 4u + r0 + i;
          qh[i] = __shfl_sync(kFull, my_hi, src);
          nd[i] = __shfl_sync(kFull, my_node, src);
        }
#pragma unroll
        for (int l = 0; l < DB; l++) {
          Quad kq[R];
#pragma unroll
          for (int i = 0; i < R; i++)
            kq[i] = ldg_quad(p.nodes_hi + static_cast<uint64_t>(nd[i]) * 16u + j * 4u);
#pragma unroll
          for (int i = 0; i < R; i++) {
            const uint32_t c = quad_count(kq[i], qh[i], sel, nib);
            if (l + 1 < DB) {
              nd[i] = nd[i] * 17u + 1u + c;
            } else if (j == static_cast<uint32_t>(r0 + i)) {
              if (DB > 1) my_node = nd[i];   // (one level: the lane's own node already)
              my_c = c;
            }
          }
        }
      }
      rank = static_cast<uint64_t>(my_node - p.internal_nodes) * 16u + my_c;
    }
#ifdef PLANB_BOUNDS_CHECK
    if (rank >= p.n_intervals) {
      report(p.status, 4u);
      rank = 0;
    }
#endif
    uint32_t w = __ldg(p.nh_tie + rank);
    const LoRef lo_src = lo_ref<MULTI>(p, seg.off + mine);
    w = settle_tie(p.nodes_hi + leaf_key0, p.nodes_lo + leaf_key0, nk, p.nh_tie, rank, w, my_hi,
                   [&lo_src, ok] { return ok ? *lo_src.ptr() : 0ull; });
    if (ok) store_out<MULTI>(p, seg.off + mine, static_cast<uint16_t>(w));
  }
}

// ------------------------------------------------------------------------------- flat
__global__ void __launch_bounds__(256) lookup_flat(const KParams p) {
  const ulonglong2* keys = p.nodes + static_cast<uint64_t>(p.internal_nodes) * 8u;
  const uint32_t nk = static_cast<uint32_t>(p.n_intervals - 1);
  auto gload = [keys](uint32_t i) { return __ldg(keys + i); };
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const Seg seg = segment(p);
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < seg.n;
       i += stride) {
    const uint64_t xh = p.xhi[seg.off + i], xl = *lo_ref<true>(p, seg.off + i).ptr();
    uint32_t rank = nk ? count_below(gload, nk, xh, xl) : 0u;
#ifdef PLANB_BOUNDS_CHECK
    if (rank >= p.n_intervals) {
      report(p.status, 8u);
      rank = 0;
    }
#endif
    store_out(p, seg.off + i, __ldg(p.values + rank));
  }
}

typedef void (*KernelFn)(const KParams);

constexpr int kInPlaceCtas = 4;   // 256-thread CTAs per SM of the in-place F16HI launch

constexpr int kMaxDepth = 10;

// db >= 0: the F16HI hybrid kernel for db levels below its index (an in-place search of another
// index than the table's own).
KernelFn kernel_for(const DevTable& t, bool multi = false, bool lazy = false, int db = -1) {
  static const KernelFn f8[kMaxDepth + 1] = {
      nullptr,            lookup_coop_f8<1>, lookup_coop_f8<2>, lookup_coop_f8<3>,
      lookup_coop_f8<4>,  lookup_coop_f8<5>, lookup_coop_f8<6>, lookup_coop_f8<7>,
      lookup_coop_f8<8>,  lookup_coop_f8<9>, lookup_coop_f8<10>};
  static const KernelFn f16[kMaxDepth + 1] = {
      nullptr,             lookup_coop_f16<1>, lookup_coop_f16<2>, lookup_coop_f16<3>,
      lookup_coop_f16<4>,  lookup_coop_f16<5>, lookup_coop_f16<6>, lookup_coop_f16<7>,
      lookup_coop_f16<8>,  lookup_coop_f16<9>, lookup_coop_f16<10>};
#define PLANB_HYB(P, L, M)                                                                       \
  {                                                                                               \
    lookup_hybrid<0, P, L, M>, lookup_hybrid<1, P, L, M>, lookup_hybrid<2, P, L, M>,              \
        lookup_hybrid<3, P, L, M>, lookup_hybrid<4, P, L, M>, lookup_hybrid<5, P, L, M>,          \
        lookup_hybrid<6, P, L, M>, lookup_hybrid<7, P, L, M>, lookup_hybrid<8, P, L, M>,          \
        lookup_hybrid<9, P, L, M>, lookup_hybrid<10, P, L, M>                                     \
  }
  // [packed][learned][multi]; the learned kernel has no multi-table form
  static const KernelFn hyb[2][2][kMaxDepth + 1] = {
      {PLANB_HYB(false, false, false), PLANB_HYB(false, true, false)},
      {PLANB_HYB(true, false, false), PLANB_HYB(true, true, false)}};
#undef PLANB_HYB
#define PLANB_HYB_MULTI(P)                                                                      \
  {                                                                                               \
    lookup_hybrid<0, P, false, true, true>, lookup_hybrid<1, P, false, true, true>,              \
        lookup_hybrid<2, P, false, true, true>, lookup_hybrid<3, P, false, true, true>,          \
        lookup_hybrid<4, P, false, true, true>, lookup_hybrid<5, P, false, true, true>,          \
        lookup_hybrid<6, P, false, true, true>, lookup_hybrid<7, P, false, true, true>,          \
        lookup_hybrid<8, P, false, true, true>, lookup_hybrid<9, P, false, true, true>,          \
        lookup_hybrid<10, P, false, true, true>                                                   \
  }
  // multi-table launches read an address's low half only on a tie (through the bucketing's
  // input positions), as the host-memory form does
  static const KernelFn hyb_multi[2][kMaxDepth + 1] = {PLANB_HYB_MULTI(false),
                                                       PLANB_HYB_MULTI(true)};
#undef PLANB_HYB_MULTI
#define PLANB_HYB_LAZY(P)                                                                       \
  {                                                                                               \
    lookup_hybrid<0, P, false, false, true>, lookup_hybrid<1, P, false, false, true>,            \
        lookup_hybrid<2, P, false, false, true>, lookup_hybrid<3, P, false, false, true>,        \
        lookup_hybrid<4, P, false, false, true>, lookup_hybrid<5, P, false, false, true>,        \
        lookup_hybrid<6, P, false, false, true>, lookup_hybrid<7, P, false, false, true>,        \
        lookup_hybrid<8, P, false, false, true>, lookup_hybrid<9, P, false, false, true>,        \
        lookup_hybrid<10, P, false, false, true>                                                  \
  }
  static const KernelFn hyb_lazy[2][kMaxDepth + 1] = {PLANB_HYB_LAZY(false), PLANB_HYB_LAZY(true)};
#undef PLANB_HYB_LAZY
  // [multi] (reads an address's low half only to settle a tie, so it serves host-resident
  // addresses too)
#define PLANB_HYB16(M)                                                                          \
  {                                                                                               \
    lookup_hybrid16<0, M>, lookup_hybrid16<1, M>, lookup_hybrid16<2, M>, lookup_hybrid16<3, M>,   \
        lookup_hybrid16<4, M>, lookup_hybrid16<5, M>, lookup_hybrid16<6, M>,                      \
        lookup_hybrid16<7, M>, lookup_hybrid16<8, M>, lookup_hybrid16<9, M>,                      \
        lookup_hybrid16<10, M>                                                                    \
  }
  static const KernelFn hyb16[2][kMaxDepth + 1] = {PLANB_HYB16(false), PLANB_HYB16(true)};
#undef PLANB_HYB16
  const uint32_t D = t.depth;
  if (D < 1 || D > static_cast<uint32_t>(kMaxDepth)) return nullptr;
  if (t.format == PLANB_FMT_F16HI && t.kernel == kHybrid && db >= 0)
    return db <= kMaxDepth ? hyb16[multi ? 1 : 0][db] : nullptr;
  if (t.format == PLANB_FMT_F16HI && t.kernel == kHybrid)
    return t.smem_levels <= D ? hyb16[multi ? 1 : 0][D - t.smem_levels] : nullptr;
  if (t.format == PLANB_FMT_F16HI) return f16[D];
  const bool packed = t.format == PLANB_FMT_F8V7;
  if (t.kernel == kHybrid && multi)
    return t.smem_levels <= D ? hyb_multi[packed][D - t.smem_levels] : nullptr;
  if (t.kernel == kHybrid && lazy)
    return t.smem_levels <= D ? hyb_lazy[packed][D - t.smem_levels] : nullptr;
  if (t.kernel == kHybrid || t.kernel == kLearned)
    return t.smem_levels <= D ? hyb[packed][t.kernel == kLearned][D - t.smem_levels] : nullptr;
  if (packed) return nullptr;
  switch (t.kernel) {
    case kFlat: return lookup_flat;
    default: return f8[D];
  }
}

// Single-table launches on this table search its index over the leaves in place (see
// launch_lookup).
bool in_place(const DevTable& t) {
  return t.kernel == kHybrid && t.format == PLANB_FMT_F16HI && t.lidx && t.lidx_db == 1;
}

}  // namespace

int kernel_attributes(const DevTable& t, bool multi, int* out) {
  KernelFn fn = kernel_for(t, multi);
  if (!multi && in_place(t)) fn = lookup_hybrid16<1, false, kInPlaceCtas>;   // what launches
  if (!fn) return PLANB_EINVAL;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(fn)) != cudaSuccess) return PLANB_ECUDA;
  out[0] = a.numRegs;
  out[1] = a.maxThreadsPerBlock;
  out[2] = a.maxDynamicSharedSizeBytes;
  out[3] = static_cast<int>(a.localSizeBytes);
  out[4] = static_cast<int>(a.sharedSizeBytes);
  out[5] = static_cast<int>(a.constSizeBytes);
  return PLANB_OK;
}

size_t smem_bytes_for(const Layout& L, uint32_t format, uint32_t levels) {
  (void)format;
  if (levels == 0) return 0;
  const uint64_t nodes = levels >= L.D ? L.total_nodes() : L.level_node[levels];
  return static_cast<size_t>(nodes) * 128u;  // both formats: 128-byte nodes
}

// Room for dynamic shared memory of a kernel: the device's opt-in maximum per block less the
// kernel's static shared memory.
int dynamic_smem_limit(const void* fn, int device, int* limit) {
  int optin = 0;
  cudaFuncAttributes a{};
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&a, fn) != cudaSuccess)
    return PLANB_ECUDA;
  *limit = optin - static_cast<int>(a.sharedSizeBytes);
  return *limit > 0 ? PLANB_OK : PLANB_EINVAL;
}

int plan_launch(const DevTable& t, int device, int threads, int ctas_per_sm, LaunchCfg& cfg) {
  KernelFn fn = kernel_for(t);
  if (!fn) return PLANB_EINVAL;
  const bool f8 = t.format != PLANB_FMT_F16HI;
  const bool hyb = (t.kernel == kHybrid || t.kernel == kLearned) && f8;
  const bool hyb16 = t.kernel == kHybrid && !f8;   // one 1024-thread CTA per SM
  const int max_threads = hyb16 ? 1024 : (hyb ? 512 : 256);
  if (threads <= 0) threads = max_threads;
  if (threads % 32 || threads > max_threads) return PLANB_EINVAL;
  cfg.threads = threads;
  if (hyb || hyb16)
    cfg.smem_bytes = static_cast<size_t>((t.sidx_n + 1) & ~1ull) * 8u +
                     (t.dir_bits ? ((((1u << t.dir_bits) + 1u) + 7u) & ~7u) * 2u : 0u) +
                     (t.kernel == kLearned ? static_cast<size_t>(t.lp.leaves) * 18u : 0u);
  else if (t.kernel == kFlat && f8)
    cfg.smem_bytes = 0;
  else
    cfg.smem_bytes = static_cast<size_t>(t.smem_nodes) * 128u;
  // The dynamic shared-memory limit is a property of the kernel function, which tables of other
  // sizes share: raise it once to the device's opt-in maximum rather than to this table's need
  // (a later, smaller table would otherwise lower it under an earlier one).
  for (KernelFn f : {fn, (t.kernel == kHybrid) ? kernel_for(t, true) : nullptr,
                     (t.kernel == kHybrid) ? kernel_for(t, false, true) : nullptr}) {
    if (!f) continue;
    int limit = 0;
    if (int rc = dynamic_smem_limit(reinterpret_cast<const void*>(f), device, &limit)) return rc;
    if (cfg.smem_bytes > static_cast<size_t>(limit)) return PLANB_EINVAL;
    if (cudaFuncSetAttribute(reinterpret_cast<const void*>(f),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess)
      return PLANB_ECUDA;
  }
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return PLANB_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(fn),
                                                    threads, cfg.smem_bytes) != cudaSuccess)
    return PLANB_ECUDA;
  if (per_sm < 1) return PLANB_EINVAL;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  cfg.blocks = sms * per_sm;
  return PLANB_OK;
}

int launch_lookup(const DevTable& t, const LaunchCfg& cfg, const uint64_t* d_hi,
                  const uint64_t* d_lo, size_t n, uint16_t* d_out, uint32_t* d_status,
                  void* stream, const uint64_t* d_range, const uint32_t* d_src,
                  bool lazy_lo) {
  if (n == 0) return PLANB_OK;
  const bool multi = d_range != nullptr;
  if (multi && t.kernel == kLearned) return PLANB_EINVAL;   // no multi-table form
  KernelFn fn = kernel_for(t, multi, lazy_lo && !multi);
  if (!fn) return PLANB_EINVAL;
  cudaGetLastError();   // the check below is about this launch, not an earlier call's leftover
  KParams p;
  p.nodes = static_cast<const ulonglong2*>(t.nodes);
  p.nodes_hi = static_cast<const uint64_t*>(t.nodes);
  p.nodes_lo = t.nodes_lo;
  p.sidx = reinterpret_cast<const ulonglong2*>(t.sidx);
  p.values = t.values;
  p.nh_tie = t.format == PLANB_FMT_F16HI ? reinterpret_cast<const uint32_t*>(t.values) : nullptr;
  p.xhi = d_hi;
  p.xlo = d_lo;
  p.out = d_out;
  p.n = n;
  p.n_intervals = t.n_intervals;
  p.total_nodes = t.total_nodes;
  p.internal_nodes = static_cast<uint32_t>(t.internal_nodes);
  p.smem_levels = t.smem_levels;
  p.smem_nodes = t.smem_nodes;
  p.sidx_n = static_cast<uint32_t>(t.sidx_n);
  p.sidx_node = static_cast<uint32_t>(t.sidx_node);
  p.status = d_status;
  p.leaves = t.leaves;
  p.leaf_err = t.leaf_err;
  p.lp = t.lp;
  p.dir = t.dir;
  p.bdir = reinterpret_cast<const ulonglong2*>(t.bdir);
  p.bdp = t.bdp;
  p.dir_bits = t.dir_bits;
  p.dir_shift = t.dir_shift;
  p.dir_base = t.dir_base;
  p.range = d_range;
  p.src = d_src;
  uint64_t blocks;
  int threads = cfg.threads;
  size_t smem = cfg.smem_bytes;
  p.staged = 1;
  // A single-table launch on an F16HI table searches its index in place, through the bucket
  // directory, rather than staging it in shared memory: its top-of-tree index when that sits right
  // above the leaves, else the leaf-level index (one L2 level below the search instead of two or
  // more). Four 256-thread CTAs per SM and no shared memory, so L1 keeps its full size for the
  // directory, index and leaf lines. Measured against the staged index: 79.5 against 79.0 B
  // lookups/s at 200 k prefixes, 77.4 against 61.8 at 1 M.
  const bool leaf = !multi && in_place(t) && cfg.blocks > 0;
  if (leaf) {
    fn = lookup_hybrid16<1, false, kInPlaceCtas>;
    p.sidx = reinterpret_cast<const ulonglong2*>(t.lidx);
    p.sidx_n = static_cast<uint32_t>(t.lidx_n);
    p.sidx_node = static_cast<uint32_t>(t.lidx_node);
    p.bdir = reinterpret_cast<const ulonglong2*>(t.lbdir);
    p.bdp = t.lbdp;
    p.dir = nullptr;
    p.dir_bits = 0;
    p.staged = 0;
    threads = 256;
    smem = 0;
    const uint64_t tiles = (n + 31) / 32;
    blocks = std::min<uint64_t>((tiles + 7) / 8, static_cast<uint64_t>(cfg.blocks) * kInPlaceCtas);
  } else if (t.kernel == kFlat) {
    blocks = (n + cfg.threads - 1) / cfg.threads;
  } else {
    const uint64_t tiles = (n + 31) / 32;
    const uint64_t warps_per_block = cfg.threads / 32;
    blocks = (tiles + warps_per_block - 1) / warps_per_block;
    // Under two tiles per warp of the full grid, staging the index would cost more than it saves:
    // search it in place, with small CTAs and no shared memory, so the launch spreads over every SM.
    const bool small = t.kernel == kHybrid && !multi && cfg.blocks > 0 &&
                       tiles < 2ull * static_cast<uint64_t>(cfg.blocks) * warps_per_block;
    if (small) {
      p.staged = 0;
      threads = 256;
      smem = 0;
      blocks = (tiles + 7) / 8;
    }
  }
  if (p.staged && cfg.blocks > 0 && blocks > static_cast<uint64_t>(cfg.blocks)) blocks = cfg.blocks;
  if (blocks == 0) blocks = 1;
  if (blocks > 65535u * 32u) blocks = 65535u * 32u;
  fn<<<static_cast<unsigned>(blocks), threads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace planb
