// Multi-table lookups (many VRF tables, one table id per address): bucketing kernels.
//
// A batch whose addresses carry a u8 table id is grouped by table with a two-pass counting sort
// over fixed chunks of the batch: each chunk's histogram (shared-memory counters), one scan that
// turns the (table, chunk) counts into output offsets in table-major order, and a scatter that
// copies each address to its table's segment and records, in input order, where it went. Each
// table's lookup then reads its segment contiguously (its table stays L2-resident while it runs)
// and writes its results contiguously in bucketed order; a final gather in input order reads each
// address's result back through the recorded position. Both the scatter's and the gather's
// scattered accesses stay local: within one chunk, a table's addresses go to one contiguous run.
// Ids at or above the table count get next hop 0 from the gather.
#include <cuda_runtime.h>

#include <cub/cub.cuh>

#include "planb_internal.h"

namespace planb {

namespace {

// batch size: from device memory when d_n is given (so one captured graph serves any size), never
// above the bound n the launch was sized for
__device__ __forceinline__ void batch_shape(const uint64_t* d_n, uint64_t& n, uint64_t& chunk) {
  if (d_n) {
    const uint64_t dn = *d_n;
    n = dn < n ? dn : n;
    chunk = n ? (n + gridDim.x - 1) / gridDim.x : 1;
  }
}

__global__ void mt_hist_kernel(const uint8_t* __restrict__ tid, uint64_t n, uint32_t T,
                               uint64_t chunk, uint32_t* __restrict__ counts /* [T+1][G] */,
                               const uint64_t* __restrict__ d_n) {
  extern __shared__ uint32_t h[];
  batch_shape(d_n, n, chunk);
  for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * chunk;
  const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  // eight independent id loads per thread per step keep enough reads in flight
  constexpr int kUnroll = 8;
  for (uint64_t i0 = b0 + threadIdx.x; i0 < b1; i0 += static_cast<uint64_t>(kUnroll) * blockDim.x) {
    uint32_t t[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; k++) {
      const uint64_t i = i0 + static_cast<uint64_t>(k) * blockDim.x;
      t[k] = i < b1 ? tid[i] : 0xFFFFu;
    }
#pragma unroll
    for (int k = 0; k < kUnroll; k++)
      if (t[k] != 0xFFFFu) atomicAdd(&h[t[k] < T ? t[k] : T], 1u);
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) counts[t * gridDim.x + blockIdx.x] = h[t];
}

// Block t scans row t of the (T+1) x G chunk counts in place into exclusive offsets within the row
// and writes the row's total.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;

__global__ void __launch_bounds__(kScanThreads) mt_rowscan_kernel(uint32_t* __restrict__ counts,
                                                                  uint32_t G,
                                                                  uint64_t* __restrict__ totals) {
  typedef cub::BlockScan<uint32_t, kScanThreads> Scan;
  __shared__ typename Scan::TempStorage tmp;
  uint32_t* row = counts + static_cast<uint64_t>(blockIdx.x) * G;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < G; base += kScanThreads * kScanItems) {
    uint32_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      const uint32_t i = base + threadIdx.x * kScanItems + k;
      v[k] = i < G ? row[i] : 0u;
    }
    uint32_t tile_total = 0;
    Scan(tmp).ExclusiveSum(v, v, tile_total);
    __syncthreads();   // tmp is reused by the next tile
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      const uint32_t i = base + threadIdx.x * kScanItems + k;
      if (i < G) row[i] = v[k] + carry;
    }
    carry += tile_total;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// One block: range[t] = sum of the totals of rows before t (range[T] starts the invalid-id
// segment, range[T+1] = the batch size).
__global__ void mt_tablescan_kernel(const uint64_t* __restrict__ totals, uint32_t T,
                                    uint64_t* __restrict__ range,
                                    unsigned long long* __restrict__ next_item) {
  typedef cub::BlockScan<uint64_t, 256> Scan;
  __shared__ typename Scan::TempStorage tmp;
  const uint32_t t = threadIdx.x;
  uint64_t v = t <= T ? totals[t] : 0ull, excl = 0, all = 0;
  Scan(tmp).ExclusiveSum(v, excl, all);
  if (t <= T) range[t] = excl;
  if (t == 0) {
    range[T + 1] = all;
    *next_item = 0ull;   // the persistent lookup that follows claims its work from here
  }
}

// The scatter works through its chunk in tiles of kTile addresses: the tile is ranked per table
// in shared memory (lanes with the same table are grouped by a warp match, so one shared atomic
// serves the group), staged in table order, and written out as one contiguous run per table, so
// the global writes are coalesced; each address's bucketed position goes to where[i] in input
// order. Positions within one table's run follow the atomics' order, not the input order: the
// recorded positions make the order immaterial.
constexpr int kScatterThreads = 256;
constexpr int kScatterItems = 8;
constexpr int kTile = kScatterThreads * kScatterItems;

__global__ void __launch_bounds__(kScatterThreads)
    mt_scatter_kernel(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                      const uint8_t* __restrict__ tid, uint64_t n, uint32_t T, uint64_t chunk,
                      const uint32_t* __restrict__ offsets, const uint64_t* __restrict__ range,
                      uint64_t* __restrict__ bhi, uint64_t* __restrict__ blo,
                      uint32_t* __restrict__ where, const uint64_t* __restrict__ d_n) {
  typedef cub::BlockScan<uint32_t, kScatterThreads> Scan;
  __shared__ typename Scan::TempStorage scan_tmp;
  __shared__ uint32_t cur[256], cnt[256], base[256];
  __shared__ uint64_t s_hi[kTile], s_lo[kTile];
  __shared__ uint8_t s_t[kTile];
  batch_shape(d_n, n, chunk);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x)
    cur[t] = static_cast<uint32_t>(range[t]) + offsets[t * gridDim.x + blockIdx.x];
  const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * chunk;
  const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  for (uint64_t tb = b0; tb < b1; tb += kTile) {
    for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    uint32_t tt[kScatterItems], rank[kScatterItems];
    uint64_t vh[kScatterItems], vl[kScatterItems];
#pragma unroll
    for (int k = 0; k < kScatterItems; k++) {
      const uint64_t e = tb + static_cast<uint64_t>(k) * kScatterThreads + threadIdx.x;
      const bool ok = e < b1;
      uint32_t t = 0xFFFFu;   // no address: a group of its own that takes no slot
      if (ok) {
        const uint32_t t0 = tid[e];
        t = t0 < T ? t0 : T;
        vh[k] = hi[e];
        vl[k] = lo[e];
      }
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, t);
      const uint32_t leader = __ffs(peers) - 1u;
      uint32_t first = 0;
      if (ok && lane == leader) first = atomicAdd(&cnt[t], __popc(peers));
      first = __shfl_sync(0xFFFFFFFFu, first, leader);
      tt[k] = t;
      rank[k] = first + __popc(peers & lt_mask);
    }
    __syncthreads();
    {
      uint32_t v = threadIdx.x <= T ? cnt[threadIdx.x] : 0u, excl = 0;
      Scan(scan_tmp).ExclusiveSum(v, excl);
      if (threadIdx.x <= T) base[threadIdx.x] = excl;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScatterItems; k++) {
      const uint64_t e = tb + static_cast<uint64_t>(k) * kScatterThreads + threadIdx.x;
      if (e < b1) {
        const uint32_t t = tt[k];
        const uint32_t slot = base[t] + rank[k];
        s_hi[slot] = vh[k];
        s_lo[slot] = vl[k];
        s_t[slot] = static_cast<uint8_t>(t);
        where[e] = cur[t] + rank[k];
      }
    }
    __syncthreads();
    const uint32_t m = static_cast<uint32_t>(b1 - tb < kTile ? b1 - tb : kTile);
    for (uint32_t slot = threadIdx.x; slot < m; slot += blockDim.x) {
      const uint32_t t = s_t[slot];
      const uint32_t pos = cur[t] + (slot - base[t]);
      bhi[pos] = s_hi[slot];
      blo[pos] = s_lo[slot];
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) cur[t] += cnt[t];
    // the next tile's first barrier orders these updates before their next use
  }
}

// out[i] = the result at the bucketed position of address i; 0 for an id beyond the tables
__global__ void mt_gather_kernel(const uint8_t* __restrict__ tid, const uint32_t* __restrict__ where,
                                 const uint16_t* __restrict__ bres, uint64_t n, uint32_t T,
                                 uint16_t* __restrict__ out, const uint64_t* __restrict__ d_n) {
  if (d_n) {
    const uint64_t dn = *d_n;
    n = dn < n ? dn : n;
  }
  // eight independent (id, position, result) chains per thread per step keep reads in flight
  constexpr int kUnroll = 8;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n;
       i0 += kUnroll * stride) {
    uint32_t w[kUnroll];
    bool v[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; k++) {
      const uint64_t i = i0 + k * stride;
      v[k] = i < n && tid[i] < T;
      w[k] = i < n ? where[i] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kUnroll; k++) {
      const uint64_t i = i0 + k * stride;
      if (i < n) out[i] = v[k] ? bres[w[k]] : static_cast<uint16_t>(0);
    }
  }
}

}  // namespace

int launch_bucketing(const uint64_t* d_hi, const uint64_t* d_lo, const uint8_t* d_tid, size_t n,
                     uint32_t T, uint32_t G, uint32_t* d_counts, uint64_t* d_range,
                     uint64_t* d_bhi, uint64_t* d_blo, uint32_t* d_where, void* stream,
                     const uint64_t* d_n) {
  if (T == 0 || T > 255 || G == 0 || n >= (uint64_t(1) << 32)) return PLANB_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();   // the check below is about these launches only
  const uint64_t chunk = n ? (n + G - 1) / G : 1;
  const size_t sh = (T + 1) * sizeof(uint32_t);
  uint64_t* totals = d_range + (T + 2);   // T + 1 words of scratch after the range
  mt_hist_kernel<<<G, 256, sh, st>>>(d_tid, n, T, chunk, d_counts, d_n);
  mt_rowscan_kernel<<<T + 1, kScanThreads, 0, st>>>(d_counts, G, totals);
  mt_tablescan_kernel<<<1, 256, 0, st>>>(
      totals, T, d_range, reinterpret_cast<unsigned long long*>(d_range + 2 * T + 3));
  mt_scatter_kernel<<<G, kScatterThreads, 0, st>>>(d_hi, d_lo, d_tid, n, T, chunk, d_counts,
                                                    d_range, d_bhi, d_blo, d_where, d_n);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int launch_gather(const uint8_t* d_tid, const uint32_t* d_where, const uint16_t* d_bres, size_t n,
                  uint32_t T, uint32_t G, uint16_t* d_out, void* stream, const uint64_t* d_n) {
  const uint64_t want = (static_cast<uint64_t>(n) + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(want < G ? (want ? want : 1) : G);
  cudaGetLastError();
  mt_gather_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_tid, d_where, d_bres,
                                                                          n, T, d_out, d_n);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace planb
