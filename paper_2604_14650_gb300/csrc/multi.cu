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
  for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const uint32_t t = tid[i];
    atomicAdd(&h[t < T ? t : T], 1u);
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) counts[t * gridDim.x + blockIdx.x] = h[t];
}

// One block: row t (table t's counts over the G chunks) becomes the chunks' output offsets;
// range[t], range[t+1] bound table t's segment (range[T], range[T+1] the invalid-id segment).
__global__ void mt_scan_kernel(uint32_t* __restrict__ counts, uint32_t G, uint32_t T,
                               uint64_t* __restrict__ range) {
  __shared__ uint64_t total[257];
  const uint32_t t = threadIdx.x;
  if (t <= T) {
    uint64_t s = 0;
    for (uint32_t b = 0; b < G; b++) {
      const uint32_t c = counts[t * G + b];
      counts[t * G + b] = static_cast<uint32_t>(s);
      s += c;
    }
    total[t] = s;
  }
  __syncthreads();
  if (t == 0) {
    uint64_t run = 0;
    for (uint32_t u = 0; u <= T; u++) {
      range[u] = run;
      run += total[u];
    }
    range[T + 1] = run;
  }
  __syncthreads();
  if (t <= T) {
    const uint32_t base = static_cast<uint32_t>(range[t]);
    for (uint32_t b = 0; b < G; b++) counts[t * G + b] += base;
  }
}

__global__ void mt_scatter_kernel(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                                  const uint8_t* __restrict__ tid, uint64_t n, uint32_t T,
                                  uint64_t chunk, const uint32_t* __restrict__ offsets,
                                  uint64_t* __restrict__ bhi, uint64_t* __restrict__ blo,
                                  uint32_t* __restrict__ where, const uint64_t* __restrict__ d_n) {
  extern __shared__ uint32_t cur[];
  batch_shape(d_n, n, chunk);
  for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x)
    cur[t] = offsets[t * gridDim.x + blockIdx.x];
  __syncthreads();
  const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * chunk;
  const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const uint32_t t0 = tid[i];
    const uint32_t pos = atomicAdd(&cur[t0 < T ? t0 : T], 1u);
    bhi[pos] = hi[i];
    blo[pos] = lo[i];
    where[i] = pos;
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
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    out[i] = tid[i] < T ? bres[where[i]] : static_cast<uint16_t>(0);
}

}  // namespace

int launch_bucketing(const uint64_t* d_hi, const uint64_t* d_lo, const uint8_t* d_tid, size_t n,
                     uint32_t T, uint32_t G, uint32_t* d_counts, uint64_t* d_range,
                     uint64_t* d_bhi, uint64_t* d_blo, uint32_t* d_where, void* stream,
                     const uint64_t* d_n) {
  if (T == 0 || T > 255 || G == 0 || n >= (uint64_t(1) << 32)) return PLANB_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t chunk = n ? (n + G - 1) / G : 1;
  const size_t sh = (T + 1) * sizeof(uint32_t);
  mt_hist_kernel<<<G, 256, sh, st>>>(d_tid, n, T, chunk, d_counts, d_n);
  mt_scan_kernel<<<1, 256, 0, st>>>(d_counts, G, T, d_range);
  mt_scatter_kernel<<<G, 256, sh, st>>>(d_hi, d_lo, d_tid, n, T, chunk, d_counts, d_bhi, d_blo,
                                        d_where, d_n);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int launch_gather(const uint8_t* d_tid, const uint32_t* d_where, const uint16_t* d_bres, size_t n,
                  uint32_t T, uint32_t G, uint16_t* d_out, void* stream, const uint64_t* d_n) {
  const uint64_t want = (static_cast<uint64_t>(n) + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(want < G ? (want ? want : 1) : G);
  mt_gather_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_tid, d_where, d_bres,
                                                                          n, T, d_out, d_n);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace planb
