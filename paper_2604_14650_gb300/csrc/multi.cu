// Multi-table lookups (many VRF tables, one table id per address): bucketing kernels.
//
// A batch whose addresses carry a u8 table id is grouped by table with a two-pass counting sort
// over fixed chunks of the batch: each chunk's histogram (shared-memory counters), one scan that
// turns the (table, chunk) counts into output offsets in table-major order, and a scatter that
// copies each address's high half to its table's segment, beside its input position (the lookup
// reads the low half from the input, through that position, only when a count needs it), and
// records, in input order, where it went. Each
// table's lookup then reads its segment contiguously (its table stays L2-resident while it runs)
// and writes its results contiguously in bucketed order; a final gather in input order reads each
// address's result back through the recorded position. Both the scatter's and the gather's
// scattered accesses stay local: within one chunk, a table's addresses go to one contiguous run.
// Ids at or above the table count get next hop 0 from the gather.
#include <cuda_runtime.h>

#include "planb_internal.h"
#include "primitives.cuh"

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
  static_assert(kScanThreads == prim::kThreads, "block scan width");
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  uint32_t* row = counts + static_cast<uint64_t>(blockIdx.x) * G;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < G; base += kScanThreads * kScanItems) {
    uint32_t v[kScanItems];
    uint32_t own = 0;   // the thread's items, then their exclusive prefixes within the thread
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      const uint32_t i = base + threadIdx.x * kScanItems + k;
      const uint32_t c = i < G ? row[i] : 0u;
      v[k] = own;
      own += c;
    }
    uint32_t tile_total = 0;
    const uint32_t before = prim::block_scan(own, prim::Sum(), warp_tot, &tile_total) - own;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      const uint32_t i = base + threadIdx.x * kScanItems + k;
      if (i < G) row[i] = v[k] + before + carry;
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
  __shared__ uint64_t warp_tot[256 / 32];
  const uint32_t t = threadIdx.x;
  uint64_t v = t <= T ? totals[t] : 0ull, all = 0;
  const uint64_t excl = prim::block_scan(v, prim::Sum(), warp_tot, &all) - v;
  if (t <= T) range[t] = excl;
  if (t == 0) {
    range[T + 1] = all;
    *next_item = 0ull;   // the persistent lookup that follows claims its work from here
  }
}

// Asynchronous global-to-shared copies (cp.async): a tile's address halves land in shared memory
// without passing through registers, one tile ahead of their use.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The scatter works through its chunk in tiles of kTile addresses: the tile is ranked per table
// in shared memory (one shared atomic per address: lanes of a warp that hit one table's counter are
// serialised by the hardware, cheaper than grouping them first with a warp match), staged in table
// order, and written out as one contiguous run per table, so the global writes are coalesced; each
// address's bucketed position goes to where[i] in input order. Positions within one table's run
// follow the atomics' order, not the input order: the recorded positions make the order
// immaterial. The tile's high and low halves are copied into
// shared memory one tile ahead (double-buffered cp.async) and its table ids read into registers
// one tile ahead, so the ranking of a tile overlaps the loads of the next; staging records for
// each slot which input address fills it, and the write reads the halves from there.
constexpr int kScatterThreads = 256;
constexpr int kScatterItems = 8;
constexpr int kTile = kScatterThreads * kScatterItems;
constexpr size_t kScatterSmem =
    2 * kTile * sizeof(uint64_t) + kTile * sizeof(uint16_t) + kTile * sizeof(uint8_t);

__global__ void __launch_bounds__(kScatterThreads)
    mt_scatter_kernel(const uint64_t* __restrict__ hi, const uint8_t* __restrict__ tid,
                      uint64_t n, uint32_t T, uint64_t chunk,
                      const uint32_t* __restrict__ offsets, const uint64_t* __restrict__ range,
                      uint64_t* __restrict__ bhi, uint32_t* __restrict__ bsrc,
                      uint16_t* __restrict__ where, uint32_t* __restrict__ tile_start,
                      uint16_t* __restrict__ tile_base, const uint64_t* __restrict__ d_n) {
  static_assert(kScatterThreads == prim::kThreads, "block scan width");
  __shared__ uint32_t scan_tot[kScatterThreads / 32];
  __shared__ uint32_t cur[256], cnt[256], base[256];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* s_in = reinterpret_cast<uint64_t*>(smem_raw);   // [buffer][kTile] high halves
  uint16_t* s_src = reinterpret_cast<uint16_t*>(s_in + 2 * kTile);   // input index per slot
  uint8_t* s_t = reinterpret_cast<uint8_t*>(s_src + kTile);           // table per slot
  batch_shape(d_n, n, chunk);
  for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x)
    cur[t] = static_cast<uint32_t>(range[t]) + offsets[t * gridDim.x + blockIdx.x];
  const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * chunk;
  const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  const uint64_t tiles_per_chunk = (chunk + kTile - 1) / kTile;
  uint64_t tile = static_cast<uint64_t>(blockIdx.x) * tiles_per_chunk;
  // copies of tile [tb, tb + kTile) into buffer b; every thread commits one group per call
  auto issue = [&](uint64_t tb, uint32_t b) {
    if (tb < b1) {
      const uint64_t m = b1 - tb < static_cast<uint64_t>(kTile) ? b1 - tb : kTile;
      uint64_t* dh = s_in + b * kTile;
      for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) cp_async8(dh + k, hi + tb + k);
    }
    cp_async_commit();
  };
  // table ids of tile tb (0xFFFF: no address, a group of its own that takes no slot)
  auto ids = [&](uint64_t tb, uint32_t (&out)[kScatterItems]) {
#pragma unroll
    for (int k = 0; k < kScatterItems; k++) {
      const uint64_t e = tb + static_cast<uint64_t>(k) * kScatterThreads + threadIdx.x;
      uint32_t t = 0xFFFFu;
      if (e < b1) {
        const uint32_t t0 = tid[e];
        t = t0 < T ? t0 : T;
      }
      out[k] = t;
    }
  };
  uint32_t tn[kScatterItems];
  issue(b0, 0);
  ids(b0, tn);
  uint32_t buf = 0;
  for (uint64_t tb = b0; tb < b1; tb += kTile, tile++, buf ^= 1u) {
    uint32_t tt[kScatterItems], rank[kScatterItems];
#pragma unroll
    for (int k = 0; k < kScatterItems; k++) tt[k] = tn[k];
    issue(tb + kTile, buf ^ 1u);   // its buffer's last readers passed the previous tile's barrier
    ids(tb + kTile, tn);
    for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScatterItems; k++)
      rank[k] = tt[k] != 0xFFFFu ? atomicAdd(&cnt[tt[k]], 1u) : 0u;
    __syncthreads();
    {
      const uint32_t v = threadIdx.x <= T ? cnt[threadIdx.x] : 0u;
      uint32_t all = 0;
      const uint32_t excl = prim::block_scan(v, prim::Sum(), scan_tot, &all) - v;
      if (threadIdx.x <= T) {
        base[threadIdx.x] = excl;
        // for the gather: where each table's run of this tile starts, in the tile and globally
        tile_start[tile * (T + 1) + threadIdx.x] = cur[threadIdx.x];
        tile_base[tile * (T + 1) + threadIdx.x] = static_cast<uint16_t>(excl);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScatterItems; k++) {
      const uint32_t local = static_cast<uint32_t>(k) * kScatterThreads + threadIdx.x;
      if (tt[k] != 0xFFFFu) {
        const uint32_t slot = base[tt[k]] + rank[k];
        s_src[slot] = static_cast<uint16_t>(local);
        s_t[slot] = static_cast<uint8_t>(tt[k]);
        where[tb + local] = static_cast<uint16_t>(slot);
      }
    }
    cp_async_wait<1>();   // this tile's copies (all groups but the newest) have landed
    __syncthreads();
    const uint32_t m = static_cast<uint32_t>(b1 - tb < kTile ? b1 - tb : kTile);
    const uint64_t* sh = s_in + buf * kTile;
    for (uint32_t slot = threadIdx.x; slot < m; slot += blockDim.x) {
      const uint32_t t = s_t[slot];
      const uint32_t pos = cur[t] + (slot - base[t]);
      const uint32_t src = s_src[slot];
      bhi[pos] = sh[src];
      bsrc[pos] = static_cast<uint32_t>(tb) + src;   // n < 2^32
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) cur[t] += cnt[t];
    // the next tile's first barrier orders these updates before their next use
  }
  cp_async_wait<0>();
}

// The gather, tile by tile in the scatter's decomposition: a tile's results are its tables' runs
// of the bucketed results (each run contiguous), read into shared memory in slot order; then
// out[i] = the result at address i's slot, coalesced in input order. Slots of ids beyond the tables
// read 0.
constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads)
    mt_gather_kernel(const uint16_t* __restrict__ where, const uint32_t* __restrict__ tile_start,
                     const uint16_t* __restrict__ tile_base, const uint16_t* __restrict__ bres,
                     uint64_t n, uint32_t T, uint64_t chunk, uint16_t* __restrict__ out,
                     const uint64_t* __restrict__ d_n) {
  __shared__ uint32_t st[256];
  __shared__ uint32_t sb[257];
  __shared__ uint16_t res[kTile];
  constexpr uint32_t kPer = kTile / kGatherThreads;   // consecutive slots per thread
  batch_shape(d_n, n, chunk);
  const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * chunk;
  const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  const uint64_t tiles_per_chunk = (chunk + kTile - 1) / kTile;
  uint64_t tile = static_cast<uint64_t>(blockIdx.x) * tiles_per_chunk;
  for (uint64_t tb = b0; tb < b1; tb += kTile, tile++) {
    const uint32_t m = static_cast<uint32_t>(b1 - tb < kTile ? b1 - tb : kTile);
    for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) {
      st[t] = tile_start[tile * (T + 1) + t];
      sb[t] = tile_base[tile * (T + 1) + t];
    }
    if (threadIdx.x == 0) sb[T + 1] = m;
    __syncthreads();
    // each thread fills kPer consecutive slots: one search for the first slot's table (the last t
    // with sb[t] <= slot; empty tables share the next table's base), then a forward walk
    const uint32_t s0 = threadIdx.x * kPer;
    if (s0 < m) {
      uint32_t lo = 0, hi = T + 1;
      while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sb[mid] <= s0) lo = mid; else hi = mid;
      }
      uint32_t t = lo;
      // the kPer source positions first (shared memory only), then their loads all in flight
      uint32_t src[kPer];
#pragma unroll
      for (uint32_t k = 0; k < kPer; k++) {
        const uint32_t slot = s0 + k;
        while (t < T + 1 && sb[t + 1] <= slot) t++;
        src[k] = (slot < m && t < T) ? st[t] + (slot - sb[t]) : 0xFFFFFFFFu;
      }
      uint16_t v[kPer];
#pragma unroll
      for (uint32_t k = 0; k < kPer; k++) v[k] = src[k] != 0xFFFFFFFFu ? bres[src[k]] : uint16_t(0);
#pragma unroll
      for (uint32_t k = 0; k < kPer; k++)
        if (s0 + k < m) res[s0 + k] = v[k];
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) out[tb + k] = res[where[tb + k]];
    __syncthreads();
  }
}

}  // namespace

int bucketing_setup() {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(mt_scatter_kernel),
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kScatterSmem)) == cudaSuccess
             ? PLANB_OK
             : PLANB_ECUDA;
}

size_t bucketing_tiles(size_t cap, uint32_t G) {
  const size_t chunk = cap ? (cap + G - 1) / G : 1;
  return static_cast<size_t>(G) * ((chunk + kTile - 1) / kTile);
}

int launch_bucketing(const uint64_t* d_hi, const uint8_t* d_tid, size_t n,
                     uint32_t T, uint32_t G, uint32_t* d_counts, uint64_t* d_range,
                     uint64_t* d_bhi, uint32_t* d_bsrc, uint16_t* d_where,
                     uint32_t* d_tile_start, uint16_t* d_tile_base, void* stream,
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
  mt_scatter_kernel<<<G, kScatterThreads, kScatterSmem, st>>>(
      d_hi, d_tid, n, T, chunk, d_counts, d_range, d_bhi, d_bsrc, d_where, d_tile_start,
      d_tile_base, d_n);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int launch_gather(const uint16_t* d_where, const uint32_t* d_tile_start,
                  const uint16_t* d_tile_base, const uint16_t* d_bres, size_t n, uint32_t T,
                  uint32_t G, uint16_t* d_out, void* stream, const uint64_t* d_n) {
  const uint64_t chunk = n ? (n + G - 1) / G : 1;
  cudaGetLastError();
  mt_gather_kernel<<<G, kGatherThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      d_where, d_tile_start, d_tile_base, d_bres, n, T, chunk, d_out, d_n);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace planb
