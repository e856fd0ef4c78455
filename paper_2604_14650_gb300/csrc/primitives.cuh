// Data-parallel primitives of the device builder, written for this library: an inclusive scan with
// any associative operator (tile scans, a scan of the tile totals, then a fix-up), a stream
// compaction by flags (a scan of the flags, then a scatter), and a stable least-significant-digit
// radix sort of (key, value) pairs in 8-bit digits (per-tile digit histograms, one scan over the
// (digit, tile) counts, then a stable scatter that ranks the equal digits of a tile with warp
// matches in tile order). All run on one stream and allocate their scratch stream-ordered.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "planb_internal.h"

namespace planb {
namespace prim {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // elements per block of every primitive
constexpr unsigned kAll = 0xFFFFFFFFu;

inline unsigned tiles_of(uint64_t n) { return static_cast<unsigned>((n + kTile - 1) / kTile); }

// Inclusive scan of the block's values, one per thread, in thread order; op need not commute.
// Returns the thread's inclusive prefix; *total receives the block's total (all threads).
template <class T, class Op>
__device__ __forceinline__ T block_scan(T v, Op op, T* warp_tot /* [kThreads / 32] */, T* total) {
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T u = __shfl_up_sync(kAll, v, d);
    if (lane >= static_cast<unsigned>(d)) v = op(u, v);
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T w = lane < kThreads / 32 ? warp_tot[lane] : warp_tot[0];
#pragma unroll
    for (int d = 1; d < kThreads / 32; d <<= 1) {
      const T u = __shfl_up_sync(kAll, w, d);
      if (lane >= static_cast<unsigned>(d)) w = op(u, w);
    }
    if (lane < kThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v = op(warp_tot[wid - 1], v);
  *total = warp_tot[kThreads / 32 - 1];
  __syncthreads();   // warp_tot may be reused by the caller
  return v;
}

struct Sum {
  template <class T>
  __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
};

// Each block scans its tile of kTile elements (thread t owns kItems consecutive ones) into out
// (which may be in: each thread reads its elements before the block's first barrier) and writes
// the tile's total to agg[block].
template <class T, class Op>
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const T* in, T* out, uint64_t n,
                                                          T* __restrict__ agg, Op op, T id) {
  __shared__ T warp_tot[kThreads / 32];
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile + threadIdx.x * kItems;
  T v[kItems];
  T run = id;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    v[k] = base + k < n ? in[base + k] : id;
    run = k == 0 ? v[k] : op(run, v[k]);
    v[k] = run;
  }
  T total;
  const T incl = block_scan(run, op, warp_tot, &total);
  // the prefix of the threads before this one: a shuffle of the inclusive results, with the
  // warp's first thread taking the previous warp's total
  T before = __shfl_up_sync(kAll, incl, 1);
  const unsigned lane = threadIdx.x & 31u;
  __shared__ T last_of_warp[kThreads / 32];
  if (lane == 31) last_of_warp[threadIdx.x >> 5] = incl;
  __syncthreads();
  if (lane == 0) before = (threadIdx.x >> 5) ? last_of_warp[(threadIdx.x >> 5) - 1] : id;
  const bool first = threadIdx.x == 0;
#pragma unroll
  for (int k = 0; k < kItems; k++)
    if (base + k < n) out[base + k] = first ? v[k] : op(before, v[k]);
  if (threadIdx.x == 0) agg[blockIdx.x] = total;
}

// out[i] = op(scanned_agg[block - 1], out[i]) for every block after the first
template <class T, class Op>
__global__ void __launch_bounds__(kThreads) k_scan_fix(T* out, uint64_t n,
                                                        const T* __restrict__ scanned_agg, Op op) {
  if (blockIdx.x == 0) return;
  const T p = scanned_agg[blockIdx.x - 1];
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile;
  for (uint32_t k = threadIdx.x; k < kTile; k += kThreads)
    if (base + k < n) out[base + k] = op(p, out[base + k]);
}

// Inclusive scan of in[0, n) into out (may alias in), on stream st.
template <class T, class Op>
int scan_inclusive(const T* in, T* out, uint64_t n, Op op, T id, cudaStream_t st) {
  if (n == 0) return PLANB_OK;
  const unsigned tiles = tiles_of(n);
  DevBuf agg;
  if (!agg.alloc(static_cast<size_t>(tiles) * sizeof(T), st)) return PLANB_ENOMEM;
  k_scan_tiles<T, Op><<<tiles, kThreads, 0, st>>>(in, out, n, agg.as<T>(), op, id);
  if (tiles > 1) {
    if (int rc = scan_inclusive<T, Op>(agg.as<T>(), agg.as<T>(), tiles, op, id, st)) return rc;
    k_scan_fix<T, Op><<<tiles, kThreads, 0, st>>>(out, n, agg.as<T>(), op);
  }
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

__global__ void k_flags_u32(const uint8_t* __restrict__ f, uint64_t n, uint32_t* __restrict__ o) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    o[i] = f[i] ? 1u : 0u;
}

template <class T>
__global__ void k_compact(const T* __restrict__ in, const uint8_t* __restrict__ f,
                          const uint32_t* __restrict__ incl, uint64_t n, T* __restrict__ out,
                          uint32_t* __restrict__ count) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    if (f[i]) out[incl[i] - 1] = in[i];
    if (i + 1 == n) *count = incl[i];
  }
}

inline unsigned grid_of(uint64_t n) {
  const uint64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<unsigned>(b < 4096 ? (b ? b : 1) : 4096);
}

// out = the entries of in[0, n) whose flag is nonzero, in order; *d_count (device) = how many.
template <class T>
int select_flagged(const T* in, const uint8_t* flags, T* out, uint64_t n, uint32_t* d_count,
                   cudaStream_t st) {
  if (n == 0) return cudaMemsetAsync(d_count, 0, 4, st) == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
  DevBuf pos;
  if (!pos.alloc(n * 4, st)) return PLANB_ENOMEM;
  k_flags_u32<<<grid_of(n), kThreads, 0, st>>>(flags, n, pos.as<uint32_t>());
  if (int rc = scan_inclusive<uint32_t, Sum>(pos.as<uint32_t>(), pos.as<uint32_t>(), n, Sum(), 0u,
                                             st))
    return rc;
  k_compact<T><<<grid_of(n), kThreads, 0, st>>>(in, flags, pos.as<uint32_t>(), n, out, d_count);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

// ---------------------------------------------------------------------------- radix sort

// counts[d * tiles + t] = elements of tile t whose digit (key >> shift) & mask is d
template <class K>
__global__ void __launch_bounds__(kThreads) k_digit_hist(const K* __restrict__ key, uint64_t n,
                                                          uint32_t shift, uint32_t mask,
                                                          uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    const uint64_t i = base + static_cast<uint64_t>(k) * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[static_cast<uint32_t>(key[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  counts[static_cast<uint64_t>(threadIdx.x) * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one digit pass. Warp w of a block takes elements [w * 32 * kItems, (w + 1) *
// 32 * kItems) of the tile in order, 32 at a time; lanes with the same digit find each other with
// a warp match, and each element's rank among the equal digits before it in the warp is the
// warp's running count for the digit plus its place among its matching lanes. The warps' counts
// are then turned into offsets in warp order, and the (digit, tile) offset of the scan places the
// tile's run of each digit: equal keys keep their input order.
template <class K>
__global__ void __launch_bounds__(kThreads) k_digit_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t n, uint32_t shift,
    uint32_t mask, const uint32_t* __restrict__ incl_counts, const uint32_t* __restrict__ counts,
    K* __restrict__ kout, uint32_t* __restrict__ vout) {
  __shared__ uint32_t wc[kThreads / 32][256];
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  for (uint32_t d = lane; d < 256; d += 32) wc[wid][d] = 0;
  __syncwarp();
  const uint64_t wbase = static_cast<uint64_t>(blockIdx.x) * kTile + wid * (32u * kItems);
  uint32_t dig[kItems], rank[kItems];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    const uint64_t i = wbase + static_cast<uint64_t>(k) * 32u + lane;
    const uint32_t d = i < n ? static_cast<uint32_t>(kin[i] >> shift) & mask : 256u;
    const unsigned peers = __match_any_sync(kAll, d);
    uint32_t r = 0;
    if (d < 256u) r = wc[wid][d] + __popc(peers & lt);
    __syncwarp();
    if (d < 256u && (peers & lt) == 0) wc[wid][d] += __popc(peers);   // the group's first lane
    __syncwarp();
    dig[k] = d;
    rank[k] = r;
  }
  __syncthreads();
  {   // per digit: the warps' counts become offsets in warp order
    uint32_t run = 0;
    const uint32_t d = threadIdx.x;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) {
      const uint32_t c = wc[w][d];
      wc[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    const uint64_t i = wbase + static_cast<uint64_t>(k) * 32u + lane;
    if (i < n) {
      const uint32_t d = dig[k];
      const uint64_t cell = static_cast<uint64_t>(d) * gridDim.x + blockIdx.x;
      const uint64_t pos = static_cast<uint64_t>(incl_counts[cell] - counts[cell]) + wc[wid][d] +
                           rank[k];
      kout[pos] = kin[i];
      vout[pos] = vin[i];
    }
  }
}

// Stable sort of (key, value) pairs by the key bits [0, end_bit), in 8-bit digits, least
// significant first. kin/vin are not modified; the result goes to kout/vout. n < 2^32.
template <class K>
int sort_pairs(const K* kin, K* kout, const uint32_t* vin, uint32_t* vout, uint64_t n,
               int end_bit, cudaStream_t st) {
  if (n == 0) return PLANB_OK;
  if (n >= (uint64_t(1) << 32) || end_bit <= 0 || end_bit > static_cast<int>(8 * sizeof(K)))
    return PLANB_EINVAL;
  const int passes = (end_bit + 7) / 8;
  const unsigned tiles = tiles_of(n);
  const uint64_t cells = 256ull * tiles;
  DevBuf tk, tv, counts, incl;
  if (!tk.alloc(n * sizeof(K), st) || !tv.alloc(n * 4, st) || !counts.alloc(cells * 4, st) ||
      !incl.alloc(cells * 4, st))
    return PLANB_ENOMEM;
  const K* sk = kin;
  const uint32_t* sv = vin;
  for (int p = 0; p < passes; p++) {
    // the last pass lands in kout/vout; the ones before alternate so that it does
    const bool to_out = ((passes - 1 - p) & 1) == 0;
    K* dk = to_out ? kout : tk.as<K>();
    uint32_t* dv = to_out ? vout : tv.as<uint32_t>();
    const uint32_t shift = 8u * p;
    const int bits = end_bit - 8 * p < 8 ? end_bit - 8 * p : 8;
    const uint32_t mask = (1u << bits) - 1u;
    k_digit_hist<K><<<tiles, kThreads, 0, st>>>(sk, n, shift, mask, counts.as<uint32_t>());
    if (int rc = scan_inclusive<uint32_t, Sum>(counts.as<uint32_t>(), incl.as<uint32_t>(), cells,
                                               Sum(), 0u, st))
      return rc;
    k_digit_scatter<K><<<tiles, kThreads, 0, st>>>(sk, sv, n, shift, mask, incl.as<uint32_t>(),
                                                   counts.as<uint32_t>(), dk, dv);
    sk = dk;
    sv = dv;
  }
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace
}  // namespace prim
}  // namespace planb
