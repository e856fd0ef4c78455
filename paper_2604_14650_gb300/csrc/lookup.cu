// Lookup kernels: descent of the linearized B+-tree for a batch of 128-bit addresses
// (hot-path steps a5-a10).
//
// The paper's search (Algorithm 1, Listing 1, Section 3.2-3.5) runs one address per core through
// D node visits, each an 8-wide SIMD compare, a popcount and the child arithmetic
// i = (k+1) i + (c+1) k. Here a node visit is spread over a lane group: lane j of an 8-lane group
// holds key j of the node (one 16-byte load; the group's 8 loads are one coalesced 128-byte line),
// compares it with the address as a 128-bit number, and the warp's ballot plus a popcount of the
// group's byte give every lane the child index c. The child of node i is node b*i + 1 + c
// (Section 3.2's child_start formula counted in nodes). Four groups serve four addresses per warp
// step; each lane owns one address of a 32-address tile, so key loads (hi, lo as 8-byte words) and
// result stores (u16) are coalesced and the query is broadcast to its group by shuffles.
//
// The first `smem_levels` levels are copied once per CTA into shared memory; deeper levels are
// read through the read-only path from L2, where the whole table stays resident (Section 2.1's
// cache-residency argument, with GB300's L2 in place of a CPU's L3). The kernel is persistent: a
// grid of a few CTAs per SM strides over the tiles.
//
// Keys are the inclusive interval ends and the count is of keys strictly below the address, so the
// popcount at the leaf is the interval index r itself and the next hop is values[r].
#include <cuda_runtime.h>

#include <cstdio>

#include "planb_internal.h"

namespace planb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct KParams {
  const ulonglong2* nodes;    // F8X128 nodes (key j of node i at nodes[i*8 + j])
  const uint64_t* nodes_hi;   // F16HI high halves (key j of node i at [i*16 + j])
  const uint64_t* nodes_lo;   // F16HI low halves
  const uint16_t* values;
  const uint64_t* xhi;
  const uint64_t* xlo;
  uint16_t* out;
  uint64_t n;
  uint64_t n_intervals;
  uint64_t total_nodes;
  uint32_t internal_nodes;
  uint32_t smem_levels;
  uint32_t smem_nodes;
  uint32_t* status;
};

// 128-bit unsigned a < x, with a = (ah, al), x = (xh, xl)
__device__ __forceinline__ bool less128(uint64_t ah, uint64_t al, uint64_t xh, uint64_t xl) {
  return (ah < xh) | ((ah == xh) & (al < xl));
}

#ifdef PLANB_BOUNDS_CHECK
__device__ __forceinline__ void report(uint32_t* status, uint32_t code) {
  if (status) atomicOr(status, code);
}
#endif

// ------------------------------------------------------------------------------- F8X128
template <int D>
__global__ void __launch_bounds__(256, 4) lookup_f8x128(const KParams p) {
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

  for (uint64_t base = warp * 32; base < p.n; base += nwarps * 32) {
    const uint64_t mine = base + lane;
    const bool ok = mine < p.n;
    const uint64_t my_hi = ok ? p.xhi[mine] : 0ull;
    const uint64_t my_lo = ok ? p.xlo[mine] : 0ull;
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
    if (ok) p.out[mine] = static_cast<uint16_t>(result);
  }
}

// ------------------------------------------------------------------------------- F16HI
// 16-lane groups, two addresses per warp step; a node is 16 high halves (one 128-byte line). A
// lane whose high half equals the address's reads the matching low half from the parallel array;
// the warp takes that branch only when some lane has such a tie.
template <int D>
__global__ void __launch_bounds__(256, 4) lookup_f16hi(const KParams p) {
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

  for (uint64_t base = warp * 32; base < p.n; base += nwarps * 32) {
    const uint64_t mine = base + lane;
    const bool ok = mine < p.n;
    const uint64_t my_hi = ok ? p.xhi[mine] : 0ull;
    const uint64_t my_lo = ok ? p.xlo[mine] : 0ull;
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
        bool lt = kh < qh;
        const bool eq = kh == qh;
        if (__any_sync(kFull, eq)) {
          if (eq) lt = __ldg(p.nodes_lo + idx) < ql;
        }
        const uint32_t m = __ballot_sync(kFull, lt);
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
      const uint32_t v = __ldg(p.values + rank);
      if (j == r) result = v;
    }
    if (ok) p.out[mine] = static_cast<uint16_t>(result);
  }
}

typedef void (*KernelFn)(const KParams);

constexpr int kMaxDepth = 10;

KernelFn kernel_for(uint32_t format, uint32_t D) {
  static const KernelFn f8[kMaxDepth + 1] = {
      nullptr,           lookup_f8x128<1>, lookup_f8x128<2>, lookup_f8x128<3>,
      lookup_f8x128<4>,  lookup_f8x128<5>, lookup_f8x128<6>, lookup_f8x128<7>,
      lookup_f8x128<8>,  lookup_f8x128<9>, lookup_f8x128<10>};
  static const KernelFn f16[kMaxDepth + 1] = {
      nullptr,          lookup_f16hi<1>, lookup_f16hi<2>, lookup_f16hi<3>,
      lookup_f16hi<4>,  lookup_f16hi<5>, lookup_f16hi<6>, lookup_f16hi<7>,
      lookup_f16hi<8>,  lookup_f16hi<9>, lookup_f16hi<10>};
  if (D < 1 || D > kMaxDepth) return nullptr;
  return format == PLANB_FMT_F16HI ? f16[D] : f8[D];
}

}  // namespace

size_t smem_bytes_for(const Layout& L, uint32_t format, uint32_t levels) {
  (void)format;
  if (levels == 0) return 0;
  const uint64_t nodes = levels >= L.D ? L.total_nodes() : L.level_node[levels];
  return static_cast<size_t>(nodes) * 128u;  // both formats: 128-byte nodes
}

int plan_launch(const DevTable& t, int device, int threads, int ctas_per_sm, LaunchCfg& cfg) {
  KernelFn fn = kernel_for(t.format, t.depth);
  if (!fn) return PLANB_EINVAL;
  if (threads <= 0) threads = 256;
  if (threads % 32 || threads > 256) return PLANB_EINVAL;
  cfg.threads = threads;
  cfg.smem_bytes = static_cast<size_t>(t.smem_nodes) * 128u;
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(fn),
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(cfg.smem_bytes)) != cudaSuccess)
    return PLANB_ECUDA;
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
                  void* stream) {
  if (n == 0) return PLANB_OK;
  KernelFn fn = kernel_for(t.format, t.depth);
  if (!fn) return PLANB_EINVAL;
  KParams p;
  p.nodes = static_cast<const ulonglong2*>(t.nodes);
  p.nodes_hi = static_cast<const uint64_t*>(t.nodes);
  p.nodes_lo = t.nodes_lo;
  p.values = t.values;
  p.xhi = d_hi;
  p.xlo = d_lo;
  p.out = d_out;
  p.n = n;
  p.n_intervals = t.n_intervals;
  p.total_nodes = t.total_nodes;
  p.internal_nodes = static_cast<uint32_t>(t.internal_nodes);
  p.smem_levels = t.smem_levels;
  p.smem_nodes = t.smem_nodes;
  p.status = d_status;
  const uint64_t tiles = (n + 31) / 32;
  const uint64_t warps_per_block = cfg.threads / 32;
  uint64_t blocks = (tiles + warps_per_block - 1) / warps_per_block;
  if (cfg.blocks > 0 && blocks > static_cast<uint64_t>(cfg.blocks)) blocks = cfg.blocks;
  fn<<<static_cast<unsigned>(blocks), cfg.threads, cfg.smem_bytes,
       static_cast<cudaStream_t>(stream)>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

}  // namespace planb
