// Multi-table lookups in one persistent launch (the lookup stage of planb_multi_lookup).
#include <cuda_runtime.h>

#include <algorithm>

#include "descent.cuh"
#include "planb_internal.h"

// multi_tiles<0, ...> keeps a level loop that never runs (its tables are resolved by the index)
#pragma nv_diag_suppress 186

namespace planb {

namespace {

// All tables of a bucketed multi-table batch in one persistent launch. The bucketed addresses are
// cut into work items of W consecutive addresses, which the CTAs claim in order from a global
// counter, so the CTAs running at one time work on a narrow window of the grouped batch and only
// two or three tables are live in L2 at once. A CTA stages the top-of-tree index (high halves) and
// radix directory of each table it meets in shared memory — keeping them while its next item is
// in the same table; an index larger than the launch's share is searched in place in global
// memory instead, through the table's bucket directory when it has one — and runs the hybrid
// descent of lookup_hybrid: phase A over the index, then
// the table's remaining DB levels from L2 by lane groups (8 lanes on F8 tables, 4 lanes with
// 32-byte loads on F16HI tables), writing each result at its bucketed position. The tile code is instantiated per (DB, format) and picked per table; depths beyond
// kMultiMaxDb take a run-time level loop. Addresses with an id beyond the tables (after range[T])
// are left to the gather that follows.
constexpr int kMultiMaxDb = 4;

template <int DB, bool PACKED>   // DB < 0: run-time depth d.db
__device__ __noinline__ void multi_tiles(const MultiDesc& d, const uint64_t* Uh,
                                         const uint16_t* Dir, uint64_t s0, uint64_t s1,
                                         const uint64_t* __restrict__ xhi,
                                         const uint64_t* __restrict__ xlo,
                                         const uint32_t* __restrict__ src,
                                         uint16_t* __restrict__ out, uint32_t* status,
                                         bool staged) {
  const ulonglong2* nodes = static_cast<const ulonglong2*>(d.nodes);
  const ulonglong2* sidx = reinterpret_cast<const ulonglong2*>(d.sidx);
  const uint32_t N = d.sidx_n;
  const uint32_t db = DB >= 0 ? static_cast<uint32_t>(DB) : d.db;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t g = lane >> 3;
  const uint32_t j = lane & 7u;
  const uint32_t gshift = g * 8u;
  const uint32_t gmask = 0xFFu << gshift;
  const uint32_t wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t base = s0 + static_cast<uint64_t>(wid) * 32u; base < s1; base += nw * 32u) {
    const uint64_t mine = base + lane;
    const bool ok = mine < s1;
    const uint64_t my_hi = ok ? xhi[mine] : 0ull;
    LazyLo my_lo(ok);   // read on a high-half tie only
    const LoRef lo_src{xlo, src, mine};
    uint32_t cnt = 0;
    if (N && staged)
      cnt = index_count(Uh, N, Dir, d.dir_bits, d.dir_shift, d.dir_base, sidx, my_hi, my_lo,
                        lo_src);
    else if (N)
      cnt = index_count_global(sidx, N, d.dir, d.dir_bits, d.dir_shift, d.dir_base, my_hi, my_lo,
                               lo_src);
    uint32_t result = 0;
    if (db == 0) {
      uint32_t rank = cnt;
#ifdef PLANB_BOUNDS_CHECK
      if (rank >= d.n_intervals) {
        report(status, 2u);
        rank = 0;
      }
#endif
      result = __ldg(d.values + rank);
    } else {
      const uint32_t my_node = d.sidx_node + cnt;
      uint64_t my_rank = 0;
#pragma unroll
      for (uint32_t r0 = 0; r0 < 8; r0 += kRounds) {
        uint64_t qh[kRounds];
        uint32_t nd[kRounds], c[kRounds];
        ulonglong2 key[kRounds];
#pragma unroll
        for (int i = 0; i < kRounds; i++) {
          const uint32_t src = gshift + r0 + i;
          qh[i] = __shfl_sync(kFull, my_hi, src);
          nd[i] = __shfl_sync(kFull, my_node, src);
        }
#pragma unroll
        for (uint32_t l = 0; l < db; l++) {
#pragma unroll
          for (int i = 0; i < kRounds; i++)
            key[i] = __ldg(nodes + static_cast<uint64_t>(nd[i]) * 8u + j);
          const bool last = l + 1 == db;
          const bool keylane = !(PACKED && last) || j < 7u;
          bool lt[kRounds], eq[kRounds];
          bool anyeq = false;
#pragma unroll
          for (int i = 0; i < kRounds; i++) {
            lt[i] = keylane & (key[i].x < qh[i]);
            eq[i] = keylane & (key[i].x == qh[i]);
            anyeq |= eq[i];
          }
          if (__any_sync(kFull, anyeq)) {
#pragma unroll
            for (int i = 0; i < kRounds; i++) {
              const uint32_t need = __ballot_sync(kFull, eq[i]) & gmask;
              if (need && j == r0 + i) my_lo.get(lo_src);
              const uint64_t ql = __shfl_sync(kFull, my_lo.v, gshift + r0 + i);
              lt[i] = lt[i] | (eq[i] & (key[i].y < ql));
            }
          }
#pragma unroll
          for (int i = 0; i < kRounds; i++) {
            c[i] = __popc(__ballot_sync(kFull, lt[i]) & gmask);
            if (!last) nd[i] = nd[i] * 9u + 1u + c[i];
          }
        }
        if (PACKED) {
          // the next hop of slot c sits in slot 7 of the same leaf line (lane 7 of the group)
#pragma unroll
          for (int i = 0; i < kRounds; i++) {
#ifdef PLANB_BOUNDS_CHECK
            if (c[i] > 6u) report(status, 4u);
#endif
            const uint32_t ci = c[i] & 7u;
            const uint64_t w = ci < 4u ? key[i].x : key[i].y;
            const uint32_t f = static_cast<uint32_t>(w >> (16u * (ci & 3u))) & 0xFFFFu;
            const uint32_t v = __shfl_sync(kFull, f, gshift + 7u);
            if (j == r0 + i) result = v;
          }
        } else {
#pragma unroll
          for (int i = 0; i < kRounds; i++) {
            uint64_t rank = static_cast<uint64_t>(nd[i] - d.internal_nodes) * 8u + c[i];
#ifdef PLANB_BOUNDS_CHECK
            if (rank >= d.n_intervals) {
              report(status, 4u);
              rank = 0;
            }
#endif
            if (j == r0 + i) my_rank = rank;
          }
        }
      }
      if (!PACKED) result = __ldg(d.values + my_rank);
    }
    if (ok) out[mine] = static_cast<uint16_t>(result);
  }
}

// The same for an F16HI table (the descent of lookup_hybrid16): every level counts high halves only,
// and the next-hop word at the count says when settle_tie must finish it.
template <int DB>   // DB < 0: run-time depth d.db
__device__ __noinline__ void multi_tiles16(const MultiDesc& d, const uint64_t* Uh,
                                           const uint16_t* Dir, uint64_t s0, uint64_t s1,
                                           const uint64_t* __restrict__ xhi,
                                           const uint64_t* __restrict__ xlo,
                                           const uint32_t* __restrict__ src,
                                           uint16_t* __restrict__ out, uint32_t* status,
                                           bool staged) {
  const uint64_t leaf_key0 = static_cast<uint64_t>(d.internal_nodes) * 16u;
  const uint64_t* keys_hi = static_cast<const uint64_t*>(d.nodes) + leaf_key0;
  const uint64_t* keys_lo = d.nodes_lo + leaf_key0;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(d.values);
  const uint64_t nk = d.n_intervals - 1;
  const uint32_t N = d.sidx_n;
  const uint32_t db = DB >= 0 ? static_cast<uint32_t>(DB) : d.db;
  const uint32_t lane = threadIdx.x & 31u;
  // 4-lane groups: lane j of group g holds keys 4j .. 4j+3 of a node (one 32-byte load)
  const uint32_t g = lane >> 2;
  const uint32_t j = lane & 3u;
  const uint32_t sel = (g >> 1) | ((4u + (g >> 1)) << 4);
  const uint32_t nib = (g & 1u) ? 0xF0F0F0F0u : 0x0F0F0F0Fu;
  const uint64_t* keys16 = static_cast<const uint64_t*>(d.nodes);
  const uint32_t wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t base = s0 + static_cast<uint64_t>(wid) * 32u; base < s1; base += nw * 32u) {
    const uint64_t mine = base + lane;
    const bool ok = mine < s1;
    const uint64_t my_hi = ok ? xhi[mine] : 0ull;
    uint32_t cnt = 0;
    if (N && staged)
      cnt = index_count_hi(Uh, N, Dir, d.dir_bits, d.dir_shift, d.dir_base, my_hi);
    else if (N && d.bdir)
      cnt = index_count_hi_bucket(reinterpret_cast<const ulonglong2*>(d.sidx),
                                  reinterpret_cast<const ulonglong2*>(d.bdir), d.bdp.bits,
                                  d.bdp.shift, d.bdp.base, my_hi);
    else if (N)
      cnt = index_count_hi_global(reinterpret_cast<const ulonglong2*>(d.sidx), N, d.dir,
                                  d.dir_bits, d.dir_shift, d.dir_base, my_hi);
    uint64_t rank = cnt;
    if (db > 0) {
      uint32_t my_node = d.sidx_node + cnt;
      uint32_t my_c = 0;
      // one level left: all four addresses of a group in flight; deeper: two at a time
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
        for (uint32_t l = 0; l < db; l++) {
          Quad kq[R];
#pragma unroll
          for (int i = 0; i < R; i++)
            kq[i] = ldg_quad(keys16 + static_cast<uint64_t>(nd[i]) * 16u + j * 4u);
#pragma unroll
          for (int i = 0; i < R; i++) {
            const uint32_t c = quad_count(kq[i], qh[i], sel, nib);
            if (l + 1 < db) {
              nd[i] = nd[i] * 17u + 1u + c;
            } else if (j == static_cast<uint32_t>(r0 + i)) {
              my_node = nd[i];
              my_c = c;
            }
          }
        }
      }
      rank = static_cast<uint64_t>(my_node - d.internal_nodes) * 16u + my_c;
    }
#ifdef PLANB_BOUNDS_CHECK
    if (rank >= d.n_intervals) {
      report(status, 4u);
      rank = 0;
    }
#endif
    uint32_t w = __ldg(words + rank);
    const LoRef lo_src{xlo, src, mine};
    w = settle_tie(keys_hi, keys_lo, nk, words, rank, w, my_hi,
                   [&lo_src, ok] { return ok ? *lo_src.ptr() : 0ull; });
    if (ok) stg_hint_u16(out + mine, static_cast<uint16_t>(w), l2_policy_evict_first());
  }
}

__global__ void __launch_bounds__(512, 2)
    lookup_multi_persistent(const MultiDesc* __restrict__ desc, uint32_t T,
                            const uint64_t* __restrict__ range, const uint64_t* __restrict__ xhi,
                            const uint64_t* __restrict__ xlo, const uint32_t* __restrict__ src,
                            uint16_t* __restrict__ out,
                            unsigned long long* __restrict__ next_item,
                            uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* R = reinterpret_cast<uint64_t*>(smem_raw);           // range[0 .. T+1]
  uint64_t* Uh = R + ((T + 3u) & ~1u);                           // the staged index
  __shared__ MultiDesc d;          // the staged table (kept in shared memory: registers are short)
  __shared__ unsigned long long item;
  for (uint32_t i = threadIdx.x; i <= T + 1u; i += blockDim.x) R[i] = range[i];
  __syncthreads();
  const uint64_t nreal = R[T];
  // items of W bucketed addresses, handed out in order: the CTAs running at one time work on a
  // narrow window of the grouped batch, so only two or three tables are live in L2 at once; W
  // shrinks with the batch so a small batch still spreads over many CTAs
  uint64_t W = (nreal / (static_cast<uint64_t>(gridDim.x) * 4u) + 511u) & ~511ull;
  W = W < 512u ? 512u : (W > 16384u ? 16384u : W);
  uint32_t staged = 0xFFFFFFFFu;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next_item, 1ull);
    __syncthreads();
    const uint64_t beg = item * W;
    __syncthreads();   // every thread has read item before thread 0 takes the next one
    if (beg >= nreal) break;
    const uint64_t end = min(beg + W, nreal);
    uint32_t lo = 0, hi = T;   // the table holding address beg: R[t] <= beg < R[t+1]
    while (hi - lo > 1u) {
      const uint32_t mid = (lo + hi) >> 1;
      if (R[mid] <= beg) lo = mid; else hi = mid;
    }
    for (uint32_t t = lo; t < T && R[t] < end; t++) {
      const uint64_t s0 = max(R[t], beg), s1 = min(R[t + 1], end);
      if (s0 >= s1) continue;
      uint16_t* Dir = reinterpret_cast<uint16_t*>(Uh + ((d.sidx_n + 1u) & ~1u));
      if (t != staged) {
        __syncthreads();   // the previous table's readers are done with Uh and d
        if (threadIdx.x == 0) d = desc[t];
        __syncthreads();
        if (d.staged) {
          Dir = reinterpret_cast<uint16_t*>(Uh + ((d.sidx_n + 1u) & ~1u));
          stage_index(Uh, reinterpret_cast<const ulonglong2*>(d.sidx), d.sidx_n, Dir, d.dir,
                      d.dir_bits ? (1u << d.dir_bits) + 1u : 0u);
        } else {
          __syncthreads();
        }
        staged = t;
      }
      const uint32_t sel = d.db <= static_cast<uint32_t>(kMultiMaxDb) ? d.db : 15u;
      const bool stage = d.staged != 0u;
      if (d.f16) {
        switch (sel) {
          case 0: multi_tiles16<0>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 1: multi_tiles16<1>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 2: multi_tiles16<2>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 3: multi_tiles16<3>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 4: multi_tiles16<4>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          default: multi_tiles16<-1>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
        }
      } else if (d.packed) {
        switch (sel) {
          case 0: multi_tiles<0, true>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 1: multi_tiles<1, true>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 2: multi_tiles<2, true>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 3: multi_tiles<3, true>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 4: multi_tiles<4, true>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          default: multi_tiles<-1, true>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
        }
      } else {
        switch (sel) {
          case 0: multi_tiles<0, false>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 1: multi_tiles<1, false>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 2: multi_tiles<2, false>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 3: multi_tiles<3, false>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          case 4: multi_tiles<4, false>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
          default: multi_tiles<-1, false>(d, Uh, Dir, s0, s1, xhi, xlo, src, out, status, stage); break;
        }
      }
    }
  }
}


// The direct multi-table lookup of F16HI tables: the batch in input order, with no bucketing.
// Each lane takes its own address and that address's table: the table's record from shared
// memory, the in-place search of its index through the bucket directory, then the one level
// below it by the 4-lane groups of lookup_hybrid16. A group's four addresses may belong to four
// tables: each hands its group the table id and the node as one word, and the group's lanes read
// that table's node array from its record. The lane then reads the next-hop word, settles a
// flagged count, and stores the result at the address's input position. An address is read once
// and its result written once, both coalesced; the tables' lines come from L2.
__global__ void __launch_bounds__(512, 2)
    lookup_multi_direct(const DirectRec* __restrict__ recs, uint32_t T,
                        const uint64_t* __restrict__ xhi, const uint64_t* __restrict__ xlo,
                        const uint8_t* __restrict__ tid, uint64_t n,
                        const uint64_t* __restrict__ d_n, uint16_t* __restrict__ out,
                        uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* rw = reinterpret_cast<ulonglong2*>(smem_raw);   // record t: words 4t .. 4t + 3
  for (uint32_t i = threadIdx.x; i < 4u * T; i += blockDim.x)
    rw[i] = reinterpret_cast<const ulonglong2*>(recs)[i];
  __syncthreads();
  if (d_n) n = min(n, *d_n);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t g = lane >> 2;
  const uint32_t j = lane & 3u;
  const uint32_t sel = (g >> 1) | ((4u + (g >> 1)) << 4);
  const uint32_t nib = (g & 1u) ? 0xF0F0F0F0u : 0x0F0F0F0Fu;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint32_t stride = gridDim.x * blockDim.x;   // whole warps of 32
  uint64_t nx_hi = 0;
  uint32_t nx_t = 0xFFu;
  {
    const uint64_t first = warp * 32 + lane;
    if (first < n) {
      nx_hi = xhi[first];
      nx_t = tid[first];
    }
  }
  for (uint64_t b0 = warp * 32; b0 < n; b0 += stride) {
    const uint64_t mine = b0 + lane;
    const bool ok = mine < n;
    const uint64_t my_hi = nx_hi;
    const uint32_t t = nx_t;
    {
      // the batch streams through L2 once: evict-first, so it does not displace table lines
      const uint64_t next = mine + stride;
      nx_hi = 0ull;
      nx_t = 0xFFu;
      if (next < n) {
        nx_hi = ldg_hint_u64(xhi + next, l2_policy_evict_first());
        nx_t = ldg_hint_u8(tid + next, l2_policy_evict_first());
      }
    }
    const bool valid = ok && t < T;
    // t << 24 | the node below the index when the table has a level there, else the index count
    uint32_t tn = 0;
    bool below = false;
    if (valid) {
      const ulonglong2 w0 = rw[4u * t], w1 = rw[4u * t + 1u];
      const uint32_t packed = static_cast<uint32_t>(w1.y);
      if (w0.y)
        tn = index_count_hi_bucket(reinterpret_cast<const ulonglong2*>(w0.x),
                                   reinterpret_cast<const ulonglong2*>(w0.y), packed & 0xFFu,
                                   (packed >> 8) & 0xFFu, w1.x, my_hi);
      below = (packed >> 16) != 0u;
      if (below) tn = (t << 24) | (tn + static_cast<uint32_t>(w1.y >> 32));
    }
    uint32_t my_c = 0;
    const uint32_t act = __ballot_sync(kFull, below);
    if (act) {
      // all four addresses of a group in flight; an address with no level below its index (or
      // no table) takes no load and counts nothing
      uint64_t qh[4];
      uint32_t an[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        qh[i] = __shfl_sync(kFull, my_hi, g * 4u + i);
        an[i] = __shfl_sync(kFull, tn, g * 4u + i);
      }
      Quad kq[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        if ((act >> (g * 4u + i)) & 1u) {
          const uint64_t* nodes = reinterpret_cast<const uint64_t*>(rw[4u * (an[i] >> 24) + 2u].x);
          kq[i] = ldg_quad_hint(nodes + static_cast<uint64_t>(an[i] & 0xFFFFFFu) * 16u + j * 4u,
                                l2_policy_evict_last());
        } else {
          kq[i] = Quad{~0ull, ~0ull, ~0ull, ~0ull};
        }
      }
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const uint32_t c = quad_count(kq[i], qh[i], sel, nib);
        if (j == static_cast<uint32_t>(i)) my_c = c;
      }
    }
    uint32_t w = 0;
    if (valid) {
      const ulonglong2 w2 = rw[4u * t + 2u], w3 = rw[4u * t + 3u];
      const uint32_t* words = reinterpret_cast<const uint32_t*>(w2.y);
      const uint32_t internal = static_cast<uint32_t>(w3.y >> 32);
      uint64_t rank = below ? static_cast<uint64_t>((tn & 0xFFFFFFu) - internal) * 16u + my_c
                            : static_cast<uint64_t>(tn);
      const uint64_t nk = static_cast<uint32_t>(w3.y);
#ifdef PLANB_BOUNDS_CHECK
      if (rank > nk) {
        report(status, 4u);
        rank = 0;
      }
#endif
      w = ldg_hint_u32(words + rank, l2_policy_evict_last());
      if (w & kTieBit) {
        const uint64_t leaf0 = static_cast<uint64_t>(internal) * 16u;
        w = settle_tie(reinterpret_cast<const uint64_t*>(w2.x) + leaf0,
                       reinterpret_cast<const uint64_t*>(w3.x) + leaf0, nk, words, rank, w, my_hi,
                       [xlo, mine] { return xlo[mine]; });
      }
    }
    if (ok) stg_hint_u16(out + mine, static_cast<uint16_t>(w), l2_policy_evict_first());
  }
}

}  // namespace

int multi_persistent_setup(int device, size_t smem_bytes, int* ctas) {
  int limit = 0, sms = 0, per_sm = 0;
  const void* fn = reinterpret_cast<const void*>(lookup_multi_persistent);
  if (int rc = dynamic_smem_limit(fn, device, &limit)) return rc;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return PLANB_ECUDA;
  if (smem_bytes > static_cast<size_t>(limit)) return PLANB_EINVAL;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess)
    return PLANB_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 512, smem_bytes) != cudaSuccess)
    return PLANB_ECUDA;
  if (per_sm < 1) return PLANB_EINVAL;
  *ctas = sms * per_sm;
  return PLANB_OK;
}

int launch_multi_persistent(const MultiDesc* d_desc, uint32_t T, const uint64_t* d_range,
                            const uint64_t* d_hi, const uint64_t* d_lo, const uint32_t* d_src,
                            uint16_t* d_out,
                            unsigned long long* d_next_item, uint32_t* d_status, int ctas,
                            size_t smem_bytes, void* stream) {
  if (T == 0 || T > 255 || ctas < 1) return PLANB_EINVAL;
  cudaGetLastError();
  lookup_multi_persistent<<<static_cast<unsigned>(ctas), 512, smem_bytes,
                            static_cast<cudaStream_t>(stream)>>>(d_desc, T, d_range, d_hi, d_lo,
                                                                 d_src, d_out, d_next_item,
                                                                 d_status);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}


int multi_direct_setup(int device, uint32_t T, int* ctas) {
  if (T == 0 || T > 255) return PLANB_EINVAL;
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, reinterpret_cast<const void*>(lookup_multi_direct), 512,
          static_cast<size_t>(T) * sizeof(DirectRec)) != cudaSuccess)
    return PLANB_ECUDA;
  if (per_sm < 1) return PLANB_EINVAL;
  *ctas = sms * per_sm;
  return PLANB_OK;
}

int launch_multi_direct(const DirectRec* d_recs, uint32_t T, const uint64_t* d_hi,
                        const uint64_t* d_lo, const uint8_t* d_tid, size_t n,
                        const uint64_t* d_n, uint16_t* d_out, uint32_t* d_status, int ctas,
                        void* stream) {
  if (T == 0 || T > 255 || ctas < 1) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  const uint64_t warps = (static_cast<uint64_t>(n) + 31) / 32;   // one tile per warp at least
  const uint64_t blocks = std::min<uint64_t>(static_cast<uint64_t>(ctas), (warps + 15) / 16);
  cudaGetLastError();
  lookup_multi_direct<<<static_cast<unsigned>(blocks), 512,
                        static_cast<size_t>(T) * sizeof(DirectRec),
                        static_cast<cudaStream_t>(stream)>>>(d_recs, T, d_hi, d_lo, d_tid, n,
                                                             d_n, d_out, d_status);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace planb
