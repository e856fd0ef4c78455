// GPU builder: build steps a1-a4 on the device.
//
// The host builder (builder.cpp) sorts on the host and sweeps Algorithm 2's stack sequentially.
// Here each step is data-parallel:
//   a1  mask host bits; a stable LSD sort of an index permutation by (length, low half, high half)
//       gives (prefix, length, input order) order; keeping the last entry of each (prefix, length)
//       run drops the earlier duplicates (the last one given wins).
//   a2  events: a start per canonical prefix and an end at P + 2^(128-L) when that is below 2^128.
//       The same stable sort orders them by (address, kind, length): at one address ends come before
//       starts, starts by ascending length (the host builder's order).
//   a3  Algorithm 2's stack, as a bracket-matching scan: the depth after each event is a prefix sum
//       of +1 (start) / -1 (end). After event e the top of the stack is the LATEST start s <= e whose
//       depth after s equals the depth after e: the top was pushed at that depth, and any later
//       start at that depth would have replaced it, while a dip below that depth in between would
//       need such a later start to come back. Events are grouped by depth with a stable sort and a
//       segmented running maximum of the start positions finds s for every e. The last event at
//       each distinct address starts an interval, with the next hop of s (0 at depth 0).
//   a4  every 16-byte slot of the node array, every top-of-tree index entry and every next hop is
//       written by a closed-form kernel straight into the table's device allocation.
// The intervals, node arrays and index are identical to the host builder's, word for word.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "planb_internal.h"
#include "primitives.cuh"

namespace planb {

DevBuf::~DevBuf() { release(); }

void DevBuf::release() {
  if (p) {
    if (stream) cudaFreeAsync(p, static_cast<cudaStream_t>(stream));
    else cudaFree(p);
  }
  p = nullptr;
  bytes = 0;
}

bool DevBuf::alloc(size_t n, void* st) {
  release();
  stream = st;
  const size_t want = n ? n : 16;
  const cudaError_t e = st ? cudaMallocAsync(&p, want, static_cast<cudaStream_t>(st))
                           : cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return false;
  }
  bytes = want;
  return true;
}

namespace {

inline unsigned blocks_for(uint64_t n) {
  const uint64_t b = (n + 255) / 256;
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(b, 1u << 20)));
}

#define GRID_LOOP(i, n)                                                                     \
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < (n); \
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)

__device__ __forceinline__ u128 top_bits_dev(int L) {
  if (L <= 0) return 0;
  if (L >= 128) return ~static_cast<u128>(0);
  return ~static_cast<u128>(0) << (128 - L);
}

// ----------------------------------------------------------------------------- a1

__global__ void k_mask(const uint64_t* hi, const uint64_t* lo, const uint8_t* len, uint64_t n,
                       uint64_t* mhi, uint64_t* mlo, uint32_t* key, uint32_t* idx) {
  GRID_LOOP(i, n) {
    const u128 p = ((static_cast<u128>(hi[i]) << 64) | lo[i]) & top_bits_dev(len[i]);
    mhi[i] = static_cast<uint64_t>(p >> 64);
    mlo[i] = static_cast<uint64_t>(p);
    key[i] = len[i];
    idx[i] = static_cast<uint32_t>(i);
  }
}

template <class T>
__global__ void k_gather(const T* src, const uint32_t* idx, uint64_t n, T* dst) {
  GRID_LOOP(i, n) dst[i] = src[idx[i]];
}

// flag the last of each (prefix, length) run of the sorted order
__global__ void k_last_of_run(const uint32_t* ord, const uint64_t* mhi, const uint64_t* mlo,
                              const uint8_t* len, uint64_t n, uint8_t* keep) {
  GRID_LOOP(i, n) {
    bool last = i + 1 == n;
    if (!last) {
      const uint32_t a = ord[i], b = ord[i + 1];
      last = mhi[a] != mhi[b] || mlo[a] != mlo[b] || len[a] != len[b];
    }
    keep[i] = last;
  }
}

__global__ void k_make_prefix(const uint32_t* sel, uint64_t N, const uint64_t* mhi,
                              const uint64_t* mlo, const uint8_t* len, const uint16_t* nh,
                              Prefix* out) {
  GRID_LOOP(j, N) {
    const uint32_t i = sel[j];
    Prefix p;
    p.p = (static_cast<u128>(mhi[i]) << 64) | mlo[i];
    p.nh = nh[i];
    p.len = len[i];
    out[j] = p;
  }
}

// ----------------------------------------------------------------------------- a2

// slot 2j: the start of canonical prefix j; slot 2j+1: its end (invalid at 2^128 and for L = 0)
__global__ void k_events(const Prefix* canon, uint64_t N, uint64_t* ehi, uint64_t* elo,
                         uint32_t* ekey, uint8_t* valid, uint32_t* slot) {
  GRID_LOOP(j, N) {
    const Prefix c = canon[j];
    const int L = c.len;
    ehi[2 * j] = static_cast<uint64_t>(c.p >> 64);
    elo[2 * j] = static_cast<uint64_t>(c.p);
    ekey[2 * j] = (1u << 8) | static_cast<uint32_t>(L);  // kind 1 (start) after kind 0, by length
    valid[2 * j] = 1;
    slot[2 * j] = static_cast<uint32_t>(2 * j);
    u128 e = 0;
    if (L > 0) e = c.p + (static_cast<u128>(1) << (128 - L));  // wraps to 0 exactly at 2^128
    ehi[2 * j + 1] = static_cast<uint64_t>(e >> 64);
    elo[2 * j + 1] = static_cast<uint64_t>(e);
    ekey[2 * j + 1] = static_cast<uint32_t>(L);           // kind 0: an end
    valid[2 * j + 1] = L > 0 && e != 0;
    slot[2 * j + 1] = static_cast<uint32_t>(2 * j + 1);
  }
}

// ----------------------------------------------------------------------------- a3

__global__ void k_delta(const uint32_t* eord, const uint32_t* ekey, uint64_t E, int* delta) {
  GRID_LOOP(i, E) delta[i] = (ekey[eord[i]] >> 8) ? 1 : -1;
}

__global__ void k_depth_key(const int* depth, uint64_t E, uint32_t* dkey, uint32_t* pos) {
  GRID_LOOP(i, E) {
    dkey[i] = static_cast<uint32_t>(depth[i]);
    pos[i] = static_cast<uint32_t>(i);
  }
}

// segmented running maximum: value = (segment head << 32) | (start position + 1, or 0)
struct SegMax {
  __device__ __forceinline__ unsigned long long operator()(unsigned long long a,
                                                           unsigned long long b) const {
    if (b >> 32) return b;
    const unsigned long long va = a & 0xFFFFFFFFull, vb = b & 0xFFFFFFFFull;
    return (a & ~0xFFFFFFFFull) | (va > vb ? va : vb);
  }
};

__global__ void k_seg_values(const uint32_t* gpos, const uint32_t* gkey, const uint32_t* eord,
                             const uint32_t* ekey, uint64_t E, unsigned long long* v) {
  GRID_LOOP(i, E) {
    const uint32_t p = gpos[i];  // position in the sorted event list
    const bool head = i == 0 || gkey[i] != gkey[i - 1];
    const bool start = (ekey[eord[p]] >> 8) != 0;
    v[i] = (static_cast<unsigned long long>(head) << 32) | (start ? p + 1ull : 0ull);
  }
}

__global__ void k_top_back(const uint32_t* gpos, const unsigned long long* scan, uint64_t E,
                           uint32_t* top) {
  GRID_LOOP(i, E) top[gpos[i]] = static_cast<uint32_t>(scan[i] & 0xFFFFFFFFull);
}

// the last event at each address opens an interval; its next hop is the top of the stack
__global__ void k_interval_ends(const uint32_t* eord, const uint64_t* ehi, const uint64_t* elo,
                                const int* depth, const uint32_t* top, const Prefix* canon,
                                uint64_t E, uint64_t* ihi, uint64_t* ilo, uint16_t* inh,
                                uint8_t* keep) {
  GRID_LOOP(i, E) {
    const uint32_t a = eord[i];
    bool last = i + 1 == E;
    if (!last) {
      const uint32_t b = eord[i + 1];
      last = ehi[a] != ehi[b] || elo[a] != elo[b];
    }
    keep[i] = last;
    ihi[i] = ehi[a];
    ilo[i] = elo[a];
    uint16_t h = 0;
    if (depth[i] > 0 && top[i] > 0) h = canon[eord[top[i] - 1] >> 1].nh;  // start slot 2j -> j
    inh[i] = h;
  }
}

// final list: an interval at address 0 (next hop 0) when no event sits there, then the event
// intervals; with merge, only those whose next hop differs from the previous one
__global__ void k_finalize(const uint64_t* chi, const uint64_t* clo, const uint16_t* cnh,
                           uint64_t M, uint32_t lead, int merge, uint64_t* ohi, uint64_t* olo,
                           uint16_t* onh, uint8_t* keep) {
  GRID_LOOP(i, M + lead) {
    uint64_t h = 0, l = 0;
    uint16_t v = 0, prev = 0;
    if (i >= lead) {
      h = chi[i - lead];
      l = clo[i - lead];
      v = cnh[i - lead];
    }
    if (i > lead) prev = cnh[i - lead - 1];  // i == lead > 0: the previous one is the lead (0)
    ohi[i] = h;
    olo[i] = l;
    onh[i] = v;
    keep[i] = i == 0 || !merge || v != prev;
  }
}

// ----------------------------------------------------------------------------- a4

struct FillGeom {
  uint64_t level_node[17];
  uint64_t child_span[17];  // leaf positions under one child of a level-l node: kl * b^(D-2-l)
  uint64_t n_keys, m, internal, total;
  uint32_t k, kl, b, D;
};

// inclusive end of interval pos (the key at leaf position pos); all-ones for padding and for the
// last interval
__device__ __forceinline__ void key_at(const uint64_t* ihi, const uint64_t* ilo, uint64_t n_keys,
                                       uint64_t m, uint64_t pos, uint64_t& h, uint64_t& l) {
  if (pos >= n_keys || pos + 1 >= m) {
    h = ~0ull;
    l = ~0ull;
    return;
  }
  const uint64_t sl = ilo[pos + 1];
  l = sl - 1;
  h = ihi[pos + 1] - (sl == 0 ? 1ull : 0ull);
}

// FMT 0: F8X128, (hi, lo) pairs, k = 8; 2: F8V7 (leaf slot 7 = packed next hops);
// 1: F16HI, split hi / lo arrays, k = 16
template <int FMT>
__global__ void k_fill_nodes(FillGeom g, const uint64_t* ihi, const uint64_t* ilo,
                             const uint16_t* inh, uint64_t* nodes, uint64_t* nodes_lo) {
  GRID_LOOP(s, g.total * g.k) {
    const uint64_t node = s / g.k;
    const uint32_t c = static_cast<uint32_t>(s - node * g.k);
    uint64_t h, l;
    if (node < g.internal) {
      uint32_t lev = 0;
      while (lev + 2 < g.D && node >= g.level_node[lev + 1]) lev++;
      const uint64_t p = node - g.level_node[lev];
      const uint64_t pos = (p * g.b + c + 1) * g.child_span[lev] - 1;
      key_at(ihi, ilo, g.n_keys, g.m, pos, h, l);
    } else {
      const uint64_t j = node - g.internal;
      if (c < g.kl) {
        key_at(ihi, ilo, g.n_keys, g.m, j * g.kl + c, h, l);
      } else {  // F8V7 slot 7: the next hops of the leaf's 7 keys
        uint64_t w[2] = {0, 0};
        for (uint32_t t = 0; t < g.kl; t++) {
          const uint64_t pos = j * g.kl + t;
          const uint64_t v = pos < g.m ? inh[pos] : 0;
          w[t / 4] |= v << (16 * (t % 4));
        }
        h = w[0];
        l = w[1];
      }
    }
    if (FMT == 1) {
      nodes[s] = h;
      nodes_lo[s] = l;
    } else {
      nodes[2 * s] = h;
      nodes[2 * s + 1] = l;
    }
  }
}

// F16HI next-hop words (nh_words): the next hop, and bit 16 when the next interval starts at a
// nonzero low half (the interval's inclusive end then has a low half other than all-ones).
__global__ void k_nh_words(uint64_t m, const uint64_t* ilo, const uint16_t* nh, uint32_t* out) {
  GRID_LOOP(i, m) {
    out[i] = nh[i] | ((i + 1 < m && ilo[i + 1] != 0) ? (1u << 16) : 0u);
  }
}

__global__ void k_fill_sidx(uint64_t n, uint64_t span, const uint64_t* ihi, const uint64_t* ilo,
                            uint64_t n_keys, uint64_t m, uint64_t* out) {
  GRID_LOOP(q, n) {
    uint64_t h, l;
    key_at(ihi, ilo, n_keys, m, (q + 1) * span - 1, h, l);
    out[2 * q] = h;
    out[2 * q + 1] = l;
  }
}

// Entries of an ascending index (2 u64 per entry, high half first) whose bucket
// (hi >> shift) - base is below b.
__device__ __forceinline__ uint64_t entries_below(const uint64_t* idx, uint64_t n, uint32_t shift,
                                                  uint64_t base, uint64_t b) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if ((idx[2 * mid] >> shift) - base < b)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_fill_dir(const uint64_t* idx, uint64_t n, uint32_t shift, uint64_t base,
                           uint64_t buckets, uint16_t* out) {
  GRID_LOOP(b, buckets + 1) out[b] = static_cast<uint16_t>(entries_below(idx, n, shift, base, b));
}

__global__ void k_fill_bucket_dir(const uint64_t* idx, uint64_t n, uint32_t shift, uint64_t base,
                                  uint64_t buckets, uint64_t* out) {
  GRID_LOOP(b, buckets) {
    const uint64_t first = entries_below(idx, n, shift, base, b);
    const uint64_t next = entries_below(idx, n, shift, base, b + 1);
    out[2 * b] = first | ((next - first) << 32);
    out[2 * b + 1] = first < n ? idx[2 * first] : ~0ull;
  }
}

// ----------------------------------------------------------------------------- sorting helpers

struct Ctx {
  cudaStream_t st;
  template <class K>
  int sort_pairs(const K* kin, K* kout, const uint32_t* vin, uint32_t* vout, uint64_t n,
                 int end_bit) {
    return prim::sort_pairs<K>(kin, kout, vin, vout, n, end_bit, st);
  }
  template <class T>
  int select(const T* in, const uint8_t* flags, T* out, uint64_t n, uint32_t* d_count) {
    return prim::select_flagged<T>(in, flags, out, n, d_count, st);
  }
  int read_count(const uint32_t* d, uint32_t& h) {
    return cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                   cudaStreamSynchronize(st) == cudaSuccess
               ? PLANB_OK
               : PLANB_ECUDA;
  }
};

// Stable sort of the permutation `ord` (n entries) by (hi, lo, key) of the entries it names:
// LSD passes by key (key_bits bits), then lo, then hi. Scratch: w32a, w32b (n words), w64a, w64b
// (n double words).
int sort_by_address(Ctx& cx, const uint64_t* hi, const uint64_t* lo, const uint32_t* key,
                    int key_bits, uint64_t n, uint32_t* ord, uint32_t* w32a, uint32_t* w32b,
                    uint64_t* w64a, uint64_t* w64b) {
  if (n == 0) return PLANB_OK;
  cudaGetLastError();   // the check at the end is about these launches only
  uint32_t* a = ord;
  uint32_t* b = w32a;
  k_gather<uint32_t><<<blocks_for(n), 256, 0, cx.st>>>(key, a, n, w32b);
  int rc = cx.sort_pairs<uint32_t>(w32b, reinterpret_cast<uint32_t*>(w64a), a, b, n, key_bits);
  if (rc) return rc;
  std::swap(a, b);
  for (const uint64_t* src : {lo, hi}) {
    k_gather<uint64_t><<<blocks_for(n), 256, 0, cx.st>>>(src, a, n, w64b);
    rc = cx.sort_pairs<unsigned long long>(reinterpret_cast<const unsigned long long*>(w64b),
                                           reinterpret_cast<unsigned long long*>(w64a), a, b, n,
                                           64);
    if (rc) return rc;
    std::swap(a, b);
  }
  if (a != ord &&
      cudaMemcpyAsync(ord, a, n * 4, cudaMemcpyDeviceToDevice, cx.st) != cudaSuccess)
    return PLANB_ECUDA;
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace

int gpu_canonicalise(const uint64_t* hi, const uint64_t* lo, const uint8_t* len,
                     const uint16_t* nh, size_t n_in, void* stream, DevBuf& d_canon,
                     uint64_t& N) {
  N = 0;
  if (n_in >= (size_t(1) << 30)) return PLANB_EINVAL;
  if (n_in && (!hi || !lo || !len || !nh)) return PLANB_EINVAL;
  for (size_t i = 0; i < n_in; i++)
    if (len[i] > 128) return PLANB_EINVAL;
  Ctx cx;
  cx.st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  const uint64_t n = n_in;
  if (n == 0) return d_canon.alloc(16, stream) ? PLANB_OK : PLANB_ENOMEM;
  DevBuf d_hi, d_lo, d_len, d_nh, mhi, mlo, key, ord, w32a, w32b, w64a, w64b, keep, sel, cnt;
  if (!d_hi.alloc(n * 8, stream) || !d_lo.alloc(n * 8, stream) || !d_len.alloc(n, stream) ||
      !d_nh.alloc(n * 2, stream) || !mhi.alloc(n * 8, stream) || !mlo.alloc(n * 8, stream) ||
      !key.alloc(n * 4, stream) || !ord.alloc(n * 4, stream) || !w32a.alloc(n * 4, stream) ||
      !w32b.alloc(n * 4, stream) || !w64a.alloc(n * 8, stream) || !w64b.alloc(n * 8, stream) ||
      !keep.alloc(n, stream) || !sel.alloc(n * 4, stream) || !cnt.alloc(16, stream))
    return PLANB_ENOMEM;
  if (cudaMemcpyAsync(d_hi.p, hi, n * 8, cudaMemcpyHostToDevice, cx.st) != cudaSuccess ||
      cudaMemcpyAsync(d_lo.p, lo, n * 8, cudaMemcpyHostToDevice, cx.st) != cudaSuccess ||
      cudaMemcpyAsync(d_len.p, len, n, cudaMemcpyHostToDevice, cx.st) != cudaSuccess ||
      cudaMemcpyAsync(d_nh.p, nh, n * 2, cudaMemcpyHostToDevice, cx.st) != cudaSuccess)
    return PLANB_ECUDA;
  k_mask<<<blocks_for(n), 256, 0, cx.st>>>(d_hi.as<uint64_t>(), d_lo.as<uint64_t>(),
                                           d_len.as<uint8_t>(), n, mhi.as<uint64_t>(),
                                           mlo.as<uint64_t>(), key.as<uint32_t>(),
                                           ord.as<uint32_t>());
  int rc = sort_by_address(cx, mhi.as<uint64_t>(), mlo.as<uint64_t>(), key.as<uint32_t>(), 8, n,
                           ord.as<uint32_t>(), w32a.as<uint32_t>(), w32b.as<uint32_t>(),
                           w64a.as<uint64_t>(), w64b.as<uint64_t>());
  if (rc) return rc;
  k_last_of_run<<<blocks_for(n), 256, 0, cx.st>>>(ord.as<uint32_t>(), mhi.as<uint64_t>(),
                                                  mlo.as<uint64_t>(), d_len.as<uint8_t>(), n,
                                                  keep.as<uint8_t>());
  if ((rc = cx.select(ord.as<uint32_t>(), keep.as<uint8_t>(), sel.as<uint32_t>(), n,
                      cnt.as<uint32_t>())))
    return rc;
  uint32_t h = 0;
  if ((rc = cx.read_count(cnt.as<uint32_t>(), h))) return rc;
  N = h;
  if (!d_canon.alloc(N * sizeof(Prefix), stream)) return PLANB_ENOMEM;
  k_make_prefix<<<blocks_for(N), 256, 0, cx.st>>>(sel.as<uint32_t>(), N, mhi.as<uint64_t>(),
                                                  mlo.as<uint64_t>(), d_len.as<uint8_t>(),
                                                  d_nh.as<uint16_t>(), d_canon.as<Prefix>());
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int gpu_sweep(const Prefix* d_canon, uint64_t N, bool merge, void* stream, GpuIntervals& out) {
  out.m = 0;
  Ctx cx;
  cx.st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (N >= (uint64_t(1) << 30)) return PLANB_EINVAL;
  const uint64_t E2 = N ? 2 * N : 1;
  DevBuf ehi, elo, ekey, evalid, slot, eord, w32a, w32b, w64a, w64b, cnt;
  if (!ehi.alloc(E2 * 8, stream) || !elo.alloc(E2 * 8, stream) || !ekey.alloc(E2 * 4, stream) ||
      !evalid.alloc(E2, stream) || !slot.alloc(E2 * 4, stream) || !eord.alloc(E2 * 4, stream) ||
      !w32a.alloc(E2 * 4, stream) || !w32b.alloc(E2 * 4, stream) || !w64a.alloc(E2 * 8, stream) ||
      !w64b.alloc(E2 * 8, stream) || !cnt.alloc(16, stream))
    return PLANB_ENOMEM;
  int rc;
  uint32_t E = 0;
  if (N) {
    // a2: events, the valid ones, sorted by (address, kind, length)
    k_events<<<blocks_for(N), 256, 0, cx.st>>>(d_canon, N, ehi.as<uint64_t>(), elo.as<uint64_t>(),
                                               ekey.as<uint32_t>(), evalid.as<uint8_t>(),
                                               slot.as<uint32_t>());
    if ((rc = cx.select(slot.as<uint32_t>(), evalid.as<uint8_t>(), eord.as<uint32_t>(), 2 * N,
                        cnt.as<uint32_t>())) ||
        (rc = cx.read_count(cnt.as<uint32_t>(), E)))
      return rc;
    if ((rc = sort_by_address(cx, ehi.as<uint64_t>(), elo.as<uint64_t>(), ekey.as<uint32_t>(), 9,
                              E, eord.as<uint32_t>(), w32a.as<uint32_t>(), w32b.as<uint32_t>(),
                              w64a.as<uint64_t>(), w64b.as<uint64_t>())))
      return rc;
  }
  // a3: depth, top of the stack after every event, one interval per distinct address
  DevBuf delta, depth, gkey, gpos, segv, segs, top, ihi, ilo, inh, keep, chi, clo, cnh;
  const uint64_t Ea = E ? E : 1;
  if (!delta.alloc(Ea * 4, stream) || !depth.alloc(Ea * 4, stream) ||
      !gkey.alloc(Ea * 4, stream) || !gpos.alloc(Ea * 4, stream) || !segv.alloc(Ea * 8, stream) ||
      !segs.alloc(Ea * 8, stream) || !top.alloc(Ea * 4, stream) || !ihi.alloc(Ea * 8, stream) ||
      !ilo.alloc(Ea * 8, stream) || !inh.alloc(Ea * 2, stream) || !keep.alloc(Ea + 1, stream) ||
      !chi.alloc(Ea * 8, stream) || !clo.alloc(Ea * 8, stream) || !cnh.alloc(Ea * 2, stream))
    return PLANB_ENOMEM;
  uint32_t M = 0;
  if (E) {
    k_delta<<<blocks_for(E), 256, 0, cx.st>>>(eord.as<uint32_t>(), ekey.as<uint32_t>(), E,
                                              delta.as<int>());
    if ((rc = prim::scan_inclusive<int, prim::Sum>(delta.as<int>(), depth.as<int>(), E,
                                                   prim::Sum(), 0, cx.st)))
      return rc;
    // group by depth (at most 129 nested prefixes: 8 bits), keeping event order inside a group
    k_depth_key<<<blocks_for(E), 256, 0, cx.st>>>(depth.as<int>(), E, w32a.as<uint32_t>(),
                                                  w32b.as<uint32_t>());
    if ((rc = cx.sort_pairs<uint32_t>(w32a.as<uint32_t>(), gkey.as<uint32_t>(),
                                      w32b.as<uint32_t>(), gpos.as<uint32_t>(), E, 8)))
      return rc;
    k_seg_values<<<blocks_for(E), 256, 0, cx.st>>>(gpos.as<uint32_t>(), gkey.as<uint32_t>(),
                                                   eord.as<uint32_t>(), ekey.as<uint32_t>(), E,
                                                   segv.as<unsigned long long>());
    if ((rc = prim::scan_inclusive<unsigned long long, SegMax>(
             segv.as<unsigned long long>(), segs.as<unsigned long long>(), E, SegMax(), 0ull,
             cx.st)))
      return rc;
    k_top_back<<<blocks_for(E), 256, 0, cx.st>>>(gpos.as<uint32_t>(),
                                                 segs.as<unsigned long long>(), E,
                                                 top.as<uint32_t>());
    k_interval_ends<<<blocks_for(E), 256, 0, cx.st>>>(
        eord.as<uint32_t>(), ehi.as<uint64_t>(), elo.as<uint64_t>(), depth.as<int>(),
        top.as<uint32_t>(), d_canon, E, ihi.as<uint64_t>(), ilo.as<uint64_t>(),
        inh.as<uint16_t>(), keep.as<uint8_t>());
    if ((rc = cx.select(ihi.as<uint64_t>(), keep.as<uint8_t>(), chi.as<uint64_t>(), E,
                        cnt.as<uint32_t>())) ||
        (rc = cx.select(ilo.as<uint64_t>(), keep.as<uint8_t>(), clo.as<uint64_t>(), E,
                        cnt.as<uint32_t>())) ||
        (rc = cx.select(inh.as<uint16_t>(), keep.as<uint8_t>(), cnh.as<uint16_t>(), E,
                        cnt.as<uint32_t>())) ||
        (rc = cx.read_count(cnt.as<uint32_t>(), M)))
      return rc;
  }
  // does an interval start at address 0? (only a start event can sit there)
  uint32_t lead = 1;
  if (M) {
    uint64_t first[2] = {1, 1};
    if (cudaMemcpyAsync(&first[0], chi.p, 8, cudaMemcpyDeviceToHost, cx.st) != cudaSuccess ||
        cudaMemcpyAsync(&first[1], clo.p, 8, cudaMemcpyDeviceToHost, cx.st) != cudaSuccess ||
        cudaStreamSynchronize(cx.st) != cudaSuccess)
      return PLANB_ECUDA;
    lead = (first[0] == 0 && first[1] == 0) ? 0 : 1;
  }
  const uint64_t T = M + lead;
  DevBuf fhi, flo, fnh, fkeep;
  if (!fhi.alloc(T * 8, stream) || !flo.alloc(T * 8, stream) || !fnh.alloc(T * 2, stream) ||
      !fkeep.alloc(T, stream) || !out.hi.alloc(T * 8, stream) || !out.lo.alloc(T * 8, stream) ||
      !out.nh.alloc(T * 2, stream))
    return PLANB_ENOMEM;
  k_finalize<<<blocks_for(T), 256, 0, cx.st>>>(chi.as<uint64_t>(), clo.as<uint64_t>(),
                                               cnh.as<uint16_t>(), M, lead, merge ? 1 : 0,
                                               fhi.as<uint64_t>(), flo.as<uint64_t>(),
                                               fnh.as<uint16_t>(), fkeep.as<uint8_t>());
  uint32_t m = 0;
  if ((rc = cx.select(fhi.as<uint64_t>(), fkeep.as<uint8_t>(), out.hi.as<uint64_t>(), T,
                      cnt.as<uint32_t>())) ||
      (rc = cx.select(flo.as<uint64_t>(), fkeep.as<uint8_t>(), out.lo.as<uint64_t>(), T,
                      cnt.as<uint32_t>())) ||
      (rc = cx.select(fnh.as<uint16_t>(), fkeep.as<uint8_t>(), out.nh.as<uint16_t>(), T,
                      cnt.as<uint32_t>())) ||
      (rc = cx.read_count(cnt.as<uint32_t>(), m)))
    return rc;
  out.m = m;
  return PLANB_OK;
}

int gpu_fill(const GpuIntervals& iv, const Layout& L, uint32_t format, uint32_t S,
             uint64_t sidx_n, void* nodes, uint64_t* nodes_lo, uint64_t* sidx, void* values,
             void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  FillGeom g{};
  for (uint32_t l = 0; l <= L.D && l < 17; l++) g.level_node[l] = L.level_node[l];
  // child_span[l] = kl * b^(D-2-l) for the internal levels l = 0 .. D-2
  for (uint32_t l = 0; l + 1 < L.D; l++) {
    uint64_t s = L.kl;
    for (uint32_t t = l; t + 2 < L.D; t++) s *= L.b;
    g.child_span[l] = s;
  }
  g.n_keys = L.n_keys;
  g.m = iv.m;
  g.internal = L.internal_nodes;
  g.total = L.total_nodes();
  g.k = L.k;
  g.kl = L.kl;
  g.b = L.b;
  g.D = L.D;
  const uint64_t slots = g.total * g.k;
  const uint64_t* ih = iv.hi.as<uint64_t>();
  const uint64_t* il = iv.lo.as<uint64_t>();
  const uint16_t* in = iv.nh.as<uint16_t>();
  uint64_t* nd = static_cast<uint64_t*>(nodes);
  if (format == PLANB_FMT_F16HI)
    k_fill_nodes<1><<<blocks_for(slots), 256, 0, st>>>(g, ih, il, in, nd, nodes_lo);
  else if (format == PLANB_FMT_F8V7)
    k_fill_nodes<2><<<blocks_for(slots), 256, 0, st>>>(g, ih, il, in, nd, nullptr);
  else
    k_fill_nodes<0><<<blocks_for(slots), 256, 0, st>>>(g, ih, il, in, nd, nullptr);
  if (sidx_n && gpu_fill_index(iv, L, S, sidx_n, sidx, stream)) return PLANB_ECUDA;
  if (format == PLANB_FMT_F16HI) {
    if (iv.m)
      k_nh_words<<<blocks_for(iv.m), 256, 0, st>>>(iv.m, il, in, static_cast<uint32_t*>(values));
  } else if (iv.m &&
             cudaMemcpyAsync(values, in, iv.m * 2, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    return PLANB_ECUDA;
  }
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int gpu_fill_index(const GpuIntervals& iv, const Layout& L, uint32_t S, uint64_t n,
                   uint64_t* out, void* stream) {
  if (!n) return PLANB_OK;
  uint64_t span = 1;   // keys under one level-S node
  if (S < L.D) {
    span = L.kl;
    for (uint32_t l = S; l + 1 < L.D; l++) span *= L.b;
  }
  k_fill_sidx<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, span, iv.hi.as<uint64_t>(), iv.lo.as<uint64_t>(), L.n_keys, iv.m, out);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int gpu_fill_dir(const uint64_t* idx, uint64_t n, const DirParams& p, uint16_t* out,
                 void* stream) {
  if (!p.bits) return PLANB_OK;
  const uint64_t buckets = uint64_t(1) << p.bits;
  k_fill_dir<<<blocks_for(buckets + 1), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      idx, n, p.shift, p.base, buckets, out);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int gpu_fill_bucket_dir(const uint64_t* idx, uint64_t n, const BucketDir& p, uint64_t* out,
                        void* stream) {
  if (!p.bits) return PLANB_OK;
  const uint64_t buckets = uint64_t(1) << p.bits;
  k_fill_bucket_dir<<<blocks_for(buckets), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      idx, n, p.shift, p.base, buckets, out);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int gpu_download(const GpuIntervals& iv, void* stream, Intervals& out) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<uint64_t> h(iv.m), l(iv.m);
  out.nh.resize(iv.m);
  if (iv.m &&
      (cudaMemcpyAsync(h.data(), iv.hi.p, iv.m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(l.data(), iv.lo.p, iv.m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(out.nh.data(), iv.nh.p, iv.m * 2, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess))
    return PLANB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PLANB_ECUDA;
  out.start.resize(iv.m);
  for (uint64_t i = 0; i < iv.m; i++) out.start[i] = mk128(h[i], l[i]);
  return PLANB_OK;
}

}  // namespace planb
