// Internal declarations of libplanb: host builder (canonicalise, event sweep, tree layout) and the
// device-side table description shared by the kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "planb.h"

namespace planb {

// ------------------------------------------------------------- learned position model (data)
// (inference and training code: learned.cuh / learned.cu)
constexpr int kMlpHidden = 16;
constexpr int kMlpParams = 3 * kMlpHidden + 1;   // trained: w1, b1, w2, b2
constexpr int kMlpWeights = kMlpParams + kMlpHidden;  // + cap (the units' fixed saturation widths)
constexpr uint16_t kLeafFallback = 0xFFFFu;       // error value that sends a leaf to the tree path

// Hidden unit h: a_h = min(max(w1[h] u + b1[h], 0), cap[h]) (a ReLU that saturates at cap[h]);
// output y = b2 + sum_h w2[h] a_h.
struct MlpWeights {
  float w1[kMlpHidden];
  float b1[kMlpHidden];
  float w2[kMlpHidden];
  float b2;
  float cap[kMlpHidden];
};

struct LeafModel {
  uint64_t base;  // high half of the leaf's first key
  float a;        // predicted rank at base
  float s;        // ranks per unit of the high half
};

// Everything a lookup needs of the model besides the leaves (passed by value to the kernel).
struct LearnedParams {
  MlpWeights mlp;
  uint64_t kmin;      // high half of the smallest key
  float inv_range;    // 1 / (kmax - kmin) of the high halves
  uint32_t leaves;    // L
  uint32_t span;      // keys per level-S subtree of the tree (the index's bucket width)
  float inv_span;     // 1 / span
  uint32_t n_keys;    // ranks are in [0, n_keys)
  uint32_t pad;
};

typedef unsigned __int128 u128;

inline u128 mk128(uint64_t hi, uint64_t lo) { return (static_cast<u128>(hi) << 64) | lo; }
inline uint64_t hi64(u128 v) { return static_cast<uint64_t>(v >> 64); }
inline uint64_t lo64(u128 v) { return static_cast<uint64_t>(v); }

// top `len` bits set, len in 0..128
inline u128 top_bits(int len) {
  if (len <= 0) return 0;
  if (len >= 128) return ~static_cast<u128>(0);
  return ~static_cast<u128>(0) << (128 - len);
}

// One canonical prefix: host bits cleared; (p, len) unique in a table.
struct Prefix {
  u128 p;
  uint16_t nh;
  uint8_t len;
};

inline bool prefix_less(const Prefix& a, const Prefix& b) {
  return a.p < b.p || (a.p == b.p && a.len < b.len);
}

// Elementary intervals: start[i] is the first address of interval i (start[0] == 0, strictly
// increasing), nh[i] its next hop.
struct Intervals {
  std::vector<u128> start;
  std::vector<uint16_t> nh;
  size_t size() const { return start.size(); }
};

// Step a1 (Section 3.1): mask host bits, drop earlier duplicates of a (prefix, len), sort by
// (prefix, len). Returns PLANB_EINVAL for len > 128.
int canonicalise(const uint64_t* hi, const uint64_t* lo, const uint8_t* len, const uint16_t* nh,
                 size_t n, std::vector<Prefix>& out);

// Steps a2-a3 (Section 3.1 "Interval Partitioning"; Algorithm 2's event list, sort and stack
// sweep) on a canonical, sorted prefix list.
void sweep(const std::vector<Prefix>& canon, bool merge_equal_nh, Intervals& out);

// Device memory owned by the host code that allocated it; with a stream the allocation and the
// free are stream-ordered (cudaMallocAsync / cudaFreeAsync), so the stream must outlive the buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void* stream = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  bool alloc(size_t n, void* stream);
  void release();
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// Elementary intervals on the device (the GPU builder's a1-a3 result): first address (hi, lo) and
// next hop of each of the m intervals.
struct GpuIntervals {
  DevBuf hi, lo, nh;
  uint64_t m = 0;
};

// GPU builder (gpu_builder.cu), all on `stream`:
//   gpu_canonicalise  step a1 of host arrays: the canonical prefix list on the device (N entries,
//                     the same list and order as canonicalise()).
//   gpu_sweep         steps a2-a3 of a canonical device list: the intervals sweep() would give.
//   gpu_fill          step a4 into a table's device allocation: the node array(s) (fill_f8x128,
//                     fill_f8v7 or fill_f16hi), the top-of-tree index of level S (fill_sidx, when
//                     sidx_n > 0) and the m next hops (F16HI: the m next-hop words of
//                     nh_words).
//   gpu_download      the intervals back to the host.
struct Layout;
int gpu_canonicalise(const uint64_t* hi, const uint64_t* lo, const uint8_t* len,
                     const uint16_t* nh, size_t n, void* stream, DevBuf& d_canon, uint64_t& N);
int gpu_sweep(const Prefix* d_canon, uint64_t N, bool merge_equal_nh, void* stream,
              GpuIntervals& out);
int gpu_fill(const GpuIntervals& iv, const Layout& L, uint32_t format, uint32_t S,
             uint64_t sidx_n, void* nodes, uint64_t* nodes_lo, uint64_t* sidx, void* values,
             void* stream);
int gpu_download(const GpuIntervals& iv, void* stream, Intervals& out);
// The index of level S alone (n entries, as fill_sidx) from the device intervals.
int gpu_fill_index(const GpuIntervals& iv, const Layout& L, uint32_t S, uint64_t n,
                   uint64_t* out, void* stream);

// Linearized B+-tree arithmetic (Section 3.2).
struct Layout {
  uint32_t k = 0, b = 0, D = 0;        // keys per internal node, fanout, levels incl. leaves
  uint32_t kl = 0;                     // keys per leaf (k, or k - 1 when the leaf line also holds
                                       // the next hops of its keys)
  uint64_t n_keys = 0;                 // real keys (m - 1 inclusive interval ends)
  uint64_t internal_nodes = 0;         // complete internal levels: sum_{l<D-1} b^l
  uint64_t leaf_capacity = 0;          // b^(D-1)
  uint64_t leaf_nodes = 0;             // allocated leaves
  uint64_t level_node[17] = {0};       // first node index of level l (leaf level = internal_nodes)
  uint64_t total_nodes() const { return internal_nodes + leaf_nodes; }
};

// Smallest D with kl * b^(D-1) >= n_keys (or depth_override); kl = 0 means kl = k. Returns
// PLANB_EINVAL when D > 16.
int make_layout(uint32_t k, uint64_t n_keys, uint32_t depth_override, Layout& L, uint32_t kl = 0);

// Step a4 for PLANB_FMT_F8X128: node-major array of (hi, lo) key pairs, k = 8 per node.
// keys are the inclusive interval ends start[i+1] - 1; padding is all-ones.
void fill_f8x128(const Intervals& iv, const Layout& L, uint64_t* nodes /* 2*8*total_nodes */);

// Step a4 for PLANB_FMT_F8V7: internal nodes as F8X128; a leaf holds 7 keys in slots 0..6 and, in
// slot 7, the 7 next hops of those keys (u16, little-endian, bytes 0..13). The keys are the
// inclusive interval ends of ALL m intervals (the last one is all-ones), so the count at a leaf is
// always 0..6 and names a slot of that same leaf. Layout L must come from make_layout(8, m, 0, L, 7).
void fill_f8v7(const Intervals& iv, const Layout& L, uint64_t* nodes /* 2*8*total_nodes */);

// Step a4 for PLANB_FMT_F16HI: node-major hi halves (16 per node) and the parallel lo halves.
void fill_f16hi(const Intervals& iv, const Layout& L, uint64_t* node_hi, uint64_t* node_lo);

// The F16HI next-hop words: word i = nh[i] | 1 << 16 when interval i has a key (i < m - 1) whose
// low half is not all-ones, i.e. when start[i+1] has a nonzero low half. The lookup counts keys
// by high half only; only such a key can be below an address that shares its high half.
void nh_words(const Intervals& iv, uint32_t* out /* m */);

// Top-of-tree index for the hybrid kernel: entry q is the largest key of the subtree of the q-th
// node on level S (the key at leaf position (q + 1) * k * b^(D-1-S) - 1), for every q whose entry
// is a real key; trailing all-padding entries are left out. Counting the entries below an address
// gives the level-S node that a descent of levels 0 .. S-1 would reach (for S = D: the keys
// themselves, and the count is the interval index). Returns the entry count.
uint64_t sidx_entries(const Layout& L, uint32_t S);
void fill_sidx(const Intervals& iv, const Layout& L, uint32_t S, uint64_t* out /* 2 per entry */);

// Radix directory over the high halves of the top-of-tree index, so that a lookup's search of
// the index starts inside the few entries that share its leading bits: entry q falls in bucket
// (hi_q >> shift) - base, and dir[b] (b = 0 .. 2^bits) is the number of entries in buckets below
// b. shift is the smallest that puts every entry in one of 2^bits buckets; bits = 0 means no
// directory (an empty index, or one too long for 16-bit positions).
struct DirParams {
  uint32_t bits = 0, shift = 0;
  uint64_t base = 0;
};
uint32_t dir_bits_for(uint64_t n);   // the directory size for an index of n entries
DirParams dir_params(const uint64_t* sidx /* 2 per entry, ascending */, uint64_t n);
// the same from the high halves of the index's first and last entries
DirParams dir_params_ends(uint64_t first_hi, uint64_t last_hi, uint64_t n);
void fill_dir(const uint64_t* sidx, uint64_t n, const DirParams& p, uint16_t* dir);
inline size_t dir_bytes(const DirParams& p) {
  return p.bits ? ((((size_t(1) << p.bits) + 1) * 2 + 127) / 128) * 128 : 0;
}

// Bucket directory for searching the index in place in global memory (launches too small to stage
// it): about four buckets per entry, bucket b = (hi >> shift) - base as above, and each bucket one
// 16-byte word — its first entry's position (low 32 bits) and entry count (high 32 bits), then the
// high half of that first entry — so that one read settles a bucket of at most one entry.
struct BucketDir {
  uint32_t bits = 0, shift = 0;
  uint64_t base = 0;
};
// extra: log2 of the buckets per entry, rounded up (2: about four buckets per entry)
BucketDir bucket_dir_params(const uint64_t* sidx /* 2 per entry */, uint64_t n,
                            uint32_t extra = 2);
BucketDir bucket_dir_params_ends(uint64_t first_hi, uint64_t last_hi, uint64_t n,
                                 uint32_t extra = 2);
inline size_t bucket_dir_bytes(const BucketDir& p) {
  return p.bits ? (size_t(1) << p.bits) * 16 : 0;
}
void fill_bucket_dir(const uint64_t* sidx, uint64_t n, const BucketDir& p, uint64_t* out);
uint32_t bucket_dir_bits_for(uint64_t n, uint32_t extra = 2);
// The radix and bucket directories of a device index of n entries (fill_dir, fill_bucket_dir on
// the device: each bucket's first entry by a lower bound over the ascending high halves).
int gpu_fill_dir(const uint64_t* idx, uint64_t n, const DirParams& p, uint16_t* out,
                 void* stream);
int gpu_fill_bucket_dir(const uint64_t* idx, uint64_t n, const BucketDir& p, uint64_t* out,
                        void* stream);

// ------------------------------------------------------------------------- device side

// Everything a lookup kernel needs about one table (device pointers).
enum Kernel : uint32_t { kCoop = 1, kHybrid = 2, kFlat = 3, kLearned = 4 };

struct DevTable {
  const void* nodes;        // F8X128: ulonglong2[total_nodes * 8]; F16HI: uint64_t[total * 16]
  const uint64_t* sidx;     // hybrid: top-of-tree index, (hi, lo) per entry
  uint64_t sidx_n;          // entries in sidx
  uint64_t sidx_node;       // first node of level S (where the hybrid's per-group phase starts)
  const uint16_t* dir;      // hybrid: radix directory over the index (dir_bits = 0: none)
  const uint64_t* bdir;     // F16HI hybrid: bucket directory of the in-place search, or null
  BucketDir bdp;
  uint32_t dir_bits, dir_shift;
  uint64_t dir_base;
  uint32_t kernel;          // Kernel
  const uint64_t* nodes_lo; // F16HI: low halves, same shape; else null
  const uint16_t* values;   // next hop per interval, n_intervals entries (F16HI: u32 next-hop
                            // words, see nh_words)
  uint64_t n_intervals;
  uint64_t total_nodes;
  uint64_t internal_nodes;
  uint32_t depth;
  uint32_t format;
  uint32_t smem_levels;     // levels staged in shared memory
  uint32_t smem_nodes;      // nodes staged (the first smem_nodes of the array)
  const LeafModel* leaves;  // learned: leaf models (device)
  const uint16_t* leaf_err; // learned: per-leaf window half-width (device)
  LearnedParams lp;         // learned: root weights and constants
  // F16HI hybrid: the index searched in place by the direct multi-table launch, which leaves at
  // most one level below it (the leaf level): the top-of-tree index itself when it does, else an
  // index of the leaf level with its own bucket directory. lidx_db: levels below it (0 or 1).
  const uint64_t* lidx = nullptr;
  uint64_t lidx_n = 0;
  uint64_t lidx_node = 0;
  uint32_t lidx_db = 0;
  const uint64_t* lbdir = nullptr;
  BucketDir lbdp;
};

struct LaunchCfg {
  int threads = 256;
  int blocks = 0;           // persistent grid size cap
  size_t smem_bytes = 0;
};

// Launches the lookup kernel for one table on `stream`. d_status may be null. With d_range (device
// [begin, end)) the launch handles addresses begin..end-1 of d_hi/d_lo instead of 0..n-1 (n then only
// sizes the grid); with d_src as well, d_lo holds the batch's low halves in input order and the low
// half of address j is d_lo[d_src[j]], read only when a count needs it. lazy_lo (hybrid tables,
// single table): read an address's low half only on a high-half tie, for addresses that live in
// host memory and cross the host link.
int launch_lookup(const DevTable& t, const LaunchCfg& cfg, const uint64_t* d_hi,
                  const uint64_t* d_lo, size_t n, uint16_t* d_out, uint32_t* d_status,
                  void* stream, const uint64_t* d_range = nullptr,
                  const uint32_t* d_src = nullptr, bool lazy_lo = false);

// One table of the single-launch multi-table kernel (F8X128, F8V7 or F16HI tables of the hybrid
// kernel).
struct MultiDesc {
  const void* nodes;         // node array
  const uint64_t* sidx;      // top-of-tree index, (hi, lo) per entry
  const uint16_t* values;    // next hop per interval
  uint32_t sidx_n;           // index entries
  uint32_t sidx_node;        // first node of level S
  uint32_t internal_nodes;
  uint32_t db;               // levels below the index, read from L2 (D - S)
  uint32_t packed;           // F8V7: next hops in the leaf line
  uint32_t dir_bits;         // radix directory over the index (0: none)
  uint64_t n_intervals;
  const uint16_t* dir;
  uint64_t dir_base;
  uint32_t dir_shift;
  uint32_t f16;              // F16HI: 17-ary nodes of high halves, low halves in nodes_lo, and
                             // values holding u32 next-hop words (see nh_words)
  uint32_t staged;           // 1: index and directory staged in shared memory; 0: searched in
                             // place in global memory (an index larger than the launch's share)
  uint32_t pad;
  const uint64_t* nodes_lo;  // F16HI low halves
  const uint64_t* bdir;      // F16HI: bucket directory of the in-place search, or null
  BucketDir bdp;
};

// The single-launch multi-table kernel: raises its shared-memory limit to the device maximum and
// returns the persistent grid size for smem_bytes of dynamic shared memory per CTA.
int multi_persistent_setup(int device, size_t smem_bytes, int* ctas);
// Looks up the bucketed addresses [0, range[T]) of d_hi against table t of d_desc for the
// addresses in [range[t], range[t+1]), writing each result at its bucketed position in d_out; the
// low half of bucketed address j, read only when a count needs it, is d_lo[d_src[j]] (d_lo in the
// batch's input order).
// Work items are claimed from *d_next_item, which must be 0 when the launch starts (the bucketing
// resets it). smem_bytes: 8 * (T + 3 rounded to even) + the largest over the tables of 8 * sidx_n
// rounded up to 16 bytes plus 2 * (2^dir_bits + 1), at most the device maximum.
int launch_multi_persistent(const MultiDesc* d_desc, uint32_t T, const uint64_t* d_range,
                            const uint64_t* d_hi, const uint64_t* d_lo, const uint32_t* d_src,
                            uint16_t* d_out,
                            unsigned long long* d_next_item, uint32_t* d_status, int ctas,
                            size_t smem_bytes, void* stream);

// One F16HI table of the direct multi-table launch, 64 bytes (four 16-byte words, read from
// shared memory by the lanes that need them):
//   word 0: the in-place index (lidx) and its bucket directory (null: no index);
//   word 1: the directory's base; bits | shift << 8 | db << 16; the first node below the index;
//   word 2: the node array (high halves) and the next-hop words;
//   word 3: the low halves; the key count and the internal node count (the tie path, the rank).
struct DirectRec {
  const uint64_t* idx;
  const uint64_t* bdir;
  uint64_t bdir_base;
  uint32_t packed;
  uint32_t idx_node;
  const uint64_t* nodes;
  const uint32_t* words;
  const uint64_t* nodes_lo;
  uint32_t nk;
  uint32_t internal_nodes;
};
static_assert(sizeof(DirectRec) == 64, "direct record layout");

// The direct multi-table kernel (multi_lookup.cu): every address of the batch looked up in input
// order against table d_tid[i] of the T records (ids >= T give 0), the results written at their
// input positions. Tables of fewer than 2^24 nodes and 2^32 intervals. n addresses, or
// min(n, *d_n) when d_n is given. multi_direct_setup returns the persistent grid size.
int multi_direct_setup(int device, uint32_t T, int* ctas);
int launch_multi_direct(const DirectRec* d_recs, uint32_t T, const uint64_t* d_hi,
                        const uint64_t* d_lo, const uint8_t* d_tid, size_t n,
                        const uint64_t* d_n, uint16_t* d_out, uint32_t* d_status, int ctas,
                        void* stream);

// Multi-table bucketing (multi.cu): groups n addresses by their u8 table id (ids >= T form one
// extra segment) into d_bhi (high halves), table-major, with d_bsrc[j] = the input position of
// bucketed address j; d_range[t] .. d_range[t+1] bound table t's
// segment; d_range has room for 2T + 4 words (then T + 1 words of scratch, then the persistent
// lookup's work counter, which is reset to 0). d_counts holds (T+1) x G words. The batch is cut
// into G chunks and each chunk into tiles of up to 2,048 addresses: d_where[i] is address i's slot
// within its tile (the tile's addresses in table order), and for tile k and table t,
// d_tile_start[k(T+1) + t] and d_tile_base[k(T+1) + t] are where the tile's run of table t starts
// in the bucketed arrays and at which slot. The tile arrays hold bucketing_tiles(n bound, G) x
// (T+1) entries. n < 2^32. With d_n the kernels read the batch size from device memory (n then
// only bounds it).
size_t bucketing_tiles(size_t cap, uint32_t G);
// Raises the scatter kernel's dynamic shared-memory limit (once per device, before any launch or
// capture of launch_bucketing).
int bucketing_setup();
int launch_bucketing(const uint64_t* d_hi, const uint8_t* d_tid, size_t n,
                     uint32_t T, uint32_t G, uint32_t* d_counts, uint64_t* d_range,
                     uint64_t* d_bhi, uint32_t* d_bsrc, uint16_t* d_where,
                     uint32_t* d_tile_start, uint16_t* d_tile_base, void* stream,
                     const uint64_t* d_n = nullptr);
// d_out[i] = the bucketed result of address i (d_bres in bucketed order), 0 for ids >= T, using
// the tile records of launch_bucketing (same n, G and d_n).
int launch_gather(const uint16_t* d_where, const uint32_t* d_tile_start,
                  const uint16_t* d_tile_base, const uint16_t* d_bres, size_t n, uint32_t T,
                  uint32_t G, uint16_t* d_out, void* stream, const uint64_t* d_n = nullptr);

// cudaFuncGetAttributes of the lookup kernel a table uses (multi: its multi-table form):
// out[0..5] = registers, max threads per block, max dynamic shared bytes, local bytes, static shared
// bytes, constant bytes.
int kernel_attributes(const DevTable& t, bool multi, int* out);

// Room for dynamic shared memory of a kernel function: the device's opt-in maximum per block less
// the function's static shared memory.
int dynamic_smem_limit(const void* fn, int device, int* limit);

// Occupancy-derived launch configuration for a table on a device.
int plan_launch(const DevTable& t, int device, int threads, int ctas_per_sm, LaunchCfg& cfg);

// Staged shared-memory bytes for `levels` levels of a table layout/format.
size_t smem_bytes_for(const Layout& L, uint32_t format, uint32_t levels);

}  // namespace planb
