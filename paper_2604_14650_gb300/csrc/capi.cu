// C ABI of libplanb (declared in include/planb.h): table objects, build and upload, lookups, and
// the rebuild-and-swap update of Section 3.6.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "learned.cuh"
#include "planb_internal.h"

using planb::u128;

namespace {

std::atomic<int> g_inject{0};  // test hook: 1 = fail the next build on the host, 2 = on the device

thread_local char g_detail[256] = "";  // detail of the last failure on this thread

// records where a call failed (and the CUDA error, if any); returns code
int fail_detail(int code, const char* where, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(g_detail, sizeof(g_detail), "%s: %s", where, cudaGetErrorString(e));
  else
    snprintf(g_detail, sizeof(g_detail), "%s", where);
  return code;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Makes `dev` current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (ok && prev >= 0) cudaSetDevice(prev);
  }
};

// A non-blocking stream for the GPU builder; declared before the buffers ordered on it, so that it
// outlives them.
struct BuildStream {
  cudaStream_t s = nullptr;
  bool make() { return cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess; }
  ~BuildStream() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
};

// One built, uploaded, immutable table.
struct Table {
  int device = 0;
  void* mem = nullptr;
  size_t bytes = 0;
  planb::Layout L;
  planb::DevTable dt{};
  planb::LaunchCfg cfg;
  uint64_t n_input = 0, n_prefixes = 0;
  double build_ms = 0, upload_ms = 0;
  uint32_t builder = 0;       // PLANB_BUILDER_* that made it
  size_t dump_bytes = 0;      // node array(s), index and next hops: the deterministic prefix of mem
  planb::LearnedBuild model;  // learned kernel only
  ~Table() {
    if (mem) {
      DeviceGuard g(device);
      cudaFree(mem);
    }
  }
};

struct Retired {
  std::shared_ptr<Table> t;
  std::vector<cudaEvent_t> events;
  bool fenced = false;
};

constexpr size_t kHostChunk = size_t(1) << 21;  // keys per chunk of planb_lookup_host
constexpr int kHostSlots = 3;

}  // namespace

struct planb_fib {
  planb_opts opts{};
  int device = 0;
  std::vector<planb::Prefix> rib;  // canonical prefix list, sorted by (prefix, len)
  std::mutex cur_mu;               // guards cur and streams
  std::shared_ptr<Table> cur;
  std::vector<cudaStream_t> streams;
  bool streams_overflow = false;
  std::mutex upd_mu;               // serialises updates, retirement and the host pipeline
  std::vector<Retired> retired;
  uint64_t version = 0;
  uint64_t withdraw_absent = 0;
  uint32_t* d_status = nullptr;
  // planb_lookup_host resources
  cudaStream_t hs[kHostSlots] = {};
  cudaEvent_t he[kHostSlots] = {};
  void* hbuf = nullptr;
};

namespace {

int check_device(int dev) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return PLANB_ENODEV;
  if (dev < 0 || dev >= count) return PLANB_EINVAL;
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return PLANB_ECUDA;
  if (major != 10 || minor != 3) return PLANB_ENODEV;  // built for sm_103a only
  return PLANB_OK;
}

constexpr size_t kSmemBudget = 96 * 1024;   // per CTA; two hybrid CTAs fit one SM
constexpr size_t kDirBudget = 16 * 1024;     // the hybrid index's radix directory (2^13 + 1 u16)
constexpr size_t kSmem16Budget = 224 * 1024; // F16HI hybrid: one CTA per SM

uint32_t auto_smem_levels(const planb::Layout& L, uint32_t format) {
  // whole tree when it is small, else the deepest prefix of levels within 64 KiB
  if (planb::smem_bytes_for(L, format, L.D) <= kSmemBudget) return L.D;
  uint32_t s = 0;
  while (s + 1 < L.D && planb::smem_bytes_for(L, format, s + 1) <= 64 * 1024) s++;
  return s;
}

// levels resolved by the hybrid kernel's shared-memory index: every key when they fit, else the
// deepest level whose subtree maxima fit
uint32_t auto_index_levels(const planb::Layout& L, size_t budget) {
  if (planb::sidx_entries(L, L.D) * 8 <= budget) return L.D;   // 8 bytes (high half) per entry
  uint32_t s = 0;
  while (s + 1 < L.D && planb::sidx_entries(L, s + 1) * 8 <= budget) s++;
  return s;
}

// Builds and uploads a table from a canonical prefix list. With the device builder the intervals
// and the node arrays are made on the GPU (gpu_builder.cu) from d_canon when it is given (the
// same list, already on the device, ordered on bs) or from an upload of canon.
int make_table(const std::vector<planb::Prefix>& canon, uint64_t n_input, const planb_opts& o,
               int device, std::shared_ptr<Table>& out, BuildStream* bs = nullptr,
               const planb::DevBuf* d_canon = nullptr) {
  auto t0 = std::chrono::steady_clock::now();
  if (g_inject.load() == 1) {
    g_inject.store(0);
    return PLANB_ENOMEM;
  }
  const bool on_dev = o.builder == PLANB_BUILDER_DEVICE;
  DeviceGuard gd(device);      // current for the whole build (outlives the stream and buffers)
  if (!gd.ok) return PLANB_ECUDA;
  BuildStream own;
  if (on_dev && !bs) {
    bs = &own;
    if (!own.make()) return fail_detail(PLANB_ECUDA, "build stream");
  }
  planb::DevBuf up;            // the canonical list, uploaded (after bs: freed on it first)
  planb::GpuIntervals giv;     // device builder: the intervals
  planb::Intervals iv;         // host builder (and the learned model): the intervals
  uint64_t m = 0;
  if (on_dev) {
    void* st = bs->s;
    const planb::Prefix* dc = d_canon ? d_canon->as<planb::Prefix>() : nullptr;
    if (!dc) {
      if (!up.alloc(canon.size() * sizeof(planb::Prefix), st)) return PLANB_ENOMEM;
      if (!canon.empty() &&
          cudaMemcpyAsync(up.p, canon.data(), canon.size() * sizeof(planb::Prefix),
                          cudaMemcpyHostToDevice, bs->s) != cudaSuccess)
        return fail_detail(PLANB_ECUDA, "builder upload");
      dc = up.as<planb::Prefix>();
    }
    int rc = planb::gpu_sweep(dc, canon.size(), o.merge_equal_nh != 0, st, giv);
    if (rc) return fail_detail(rc, "device interval sweep", cudaGetLastError());
    m = giv.m;
  } else {
    planb::sweep(canon, o.merge_equal_nh != 0, iv);
    m = iv.size();
  }
  const uint32_t format = static_cast<uint32_t>(o.format);
  const uint32_t k = format == PLANB_FMT_F16HI ? 16 : 8;
  uint32_t kernel = static_cast<uint32_t>(o.kernel);
  if (kernel == PLANB_KERNEL_AUTO) kernel = planb::kHybrid;
  const bool learned = kernel == planb::kLearned;
  if (on_dev && learned) {  // the model is fitted from the host copy of the intervals
    int rc = planb::gpu_download(giv, bs->s, iv);
    if (rc) return rc;
  }
  auto t = std::make_shared<Table>();
  t->builder = on_dev ? PLANB_BUILDER_DEVICE : PLANB_BUILDER_HOST;
  t->device = device;
  t->n_input = n_input;
  t->n_prefixes = canon.size();
  // F8V7 indexes all m inclusive ends (the last is all-ones); the others the m - 1 finite ones
  int rc = format == PLANB_FMT_F8V7 ? planb::make_layout(8, m, 0, t->L, 7)
                                    : planb::make_layout(k, m - 1, 0, t->L);
  if (rc) return rc;
  const uint64_t total = t->L.total_nodes();
  if (t->L.D > 10 || total >= (uint64_t(1) << 32)) return PLANB_EINVAL;
  // levels resolved in shared memory
  uint32_t s;
  uint32_t model_leaves = 0;
  if (learned) {
    // leaf models: about one per 128 keys, a power of two in [64, 2048], then the index gets the
    // rest of the shared-memory budget; a table of a million keys or more gets 4096 (past about
    // 512 keys per leaf a line no longer keeps every rank within the 64-rank window: at 1M
    // prefixes, 2048 leaves recorded a largest bound of 88 ranks, 4096 leaves 63; 74 KB of shared
    // memory, still two CTAs per SM)
    uint32_t want = o.model_leaves > 0 ? static_cast<uint32_t>(o.model_leaves) : 64u;
    if (o.model_leaves <= 0) {
      while (want < 2048u && static_cast<uint64_t>(want) * 128u < m) want <<= 1;
      if (want == 2048u && m >= (uint64_t(1) << 20)) want = 4096u;
    }
    model_leaves = std::min<uint32_t>(want, 8192u);
    const size_t leaf_bytes = static_cast<size_t>(model_leaves) * 18u;
    const size_t budget = kSmemBudget > leaf_bytes + 8192 ? kSmemBudget - leaf_bytes : 8192;
    s = o.smem_levels < 0 ? auto_index_levels(t->L, budget)
                          : std::min<uint32_t>(o.smem_levels, t->L.D);
    while (s > 0 && planb::sidx_entries(t->L, s) * 8 + leaf_bytes > 200 * 1024) s--;
  } else if (kernel == planb::kHybrid) {
    // the index shares the budget with its radix directory (at most 16 KB); the F16HI form runs
    // one CTA per SM and may take nearly all of its shared memory
    const size_t budget = format == PLANB_FMT_F16HI ? kSmem16Budget : kSmemBudget;
    s = o.smem_levels < 0 ? auto_index_levels(t->L, budget - kDirBudget)
                          : std::min<uint32_t>(o.smem_levels, t->L.D);
    while (s > 0 && planb::sidx_entries(t->L, s) * 8 > budget - kDirBudget) s--;
  } else if (kernel == planb::kFlat) {
    s = 0;
  } else {
    s = o.smem_levels < 0 ? auto_smem_levels(t->L, format)
                          : std::min<uint32_t>(o.smem_levels, t->L.D);
    while (s > 0 && planb::smem_bytes_for(t->L, format, s) > 200 * 1024) s--;
  }
  const uint64_t sidx_n =
      (kernel == planb::kHybrid || learned) ? planb::sidx_entries(t->L, s) : 0;
  const size_t node_bytes = static_cast<size_t>(total) * 128;
  const size_t lo_bytes = format == PLANB_FMT_F16HI ? node_bytes : 0;
  const size_t sidx_bytes = ((sidx_n * 16 + 127) / 128) * 128;
  // radix directory of the hybrid index: its size depends on the entry count only
  planb::DirParams dp;
  if (kernel == planb::kHybrid) dp.bits = planb::dir_bits_for(sidx_n);
  const size_t dirb = planb::dir_bytes(dp);
  // F16HI hybrid: the bucket directory of the in-place index search (small launches); its size
  // follows from the entry count, its contents from the index
  planb::BucketDir bdp;
  if (kernel == planb::kHybrid && format == PLANB_FMT_F16HI) bdp.bits = planb::bucket_dir_bits_for(sidx_n);
  const size_t bdb = planb::bucket_dir_bytes(bdp);
  // F16HI hybrid with two or more levels below its index: an index of the leaf level too, with a
  // bucket directory of about four buckets per entry, for the in-place searches of single-table
  // and multi-table launches (one L2 level below the search instead of two or more; two buckets
  // per entry measured 77.8 against 80.2 B lookups/s at 1 M prefixes)
  const bool f16hyb = kernel == planb::kHybrid && format == PLANB_FMT_F16HI;
  const uint64_t lidx_n =
      (f16hyb && s + 1 < t->L.D) ? planb::sidx_entries(t->L, t->L.D - 1) : 0;
  const size_t lidx_bytes = ((lidx_n * 16 + 127) / 128) * 128;
  planb::BucketDir lbp;
  if (lidx_n) lbp.bits = planb::bucket_dir_bits_for(lidx_n, 2);
  const size_t lbdb = planb::bucket_dir_bytes(lbp);
  const size_t lidx_off = node_bytes + lo_bytes + sidx_bytes + dirb + bdb;
  // next hops: u16 per interval; F16HI: u32 words that also flag possible high-half ties
  const size_t vw = format == PLANB_FMT_F16HI ? 4 : 2;
  const size_t val_bytes = ((static_cast<size_t>(m) * vw + 255) / 256) * 256;
  const size_t model_bytes =
      learned ? ((static_cast<size_t>(model_leaves) * 18 + 255) / 256) * 256 : 0;
  std::vector<uint64_t> host;
  if (!on_dev) {
    host.resize((lidx_off + lidx_bytes + lbdb) / 8);
    if (format == PLANB_FMT_F16HI)
      planb::fill_f16hi(iv, t->L, host.data(), host.data() + node_bytes / 8);
    else if (format == PLANB_FMT_F8V7)
      planb::fill_f8v7(iv, t->L, host.data());
    else
      planb::fill_f8x128(iv, t->L, host.data());
    if (sidx_n) planb::fill_sidx(iv, t->L, s, host.data() + (node_bytes + lo_bytes) / 8);
    if (dp.bits) {
      const uint64_t* sx = host.data() + (node_bytes + lo_bytes) / 8;
      const uint32_t bits = dp.bits;
      dp = planb::dir_params(sx, sidx_n);
      if (dp.bits != bits) return fail_detail(PLANB_EINVAL, "radix directory size");
      planb::fill_dir(sx, sidx_n, dp, reinterpret_cast<uint16_t*>(
                                          host.data() + (node_bytes + lo_bytes + sidx_bytes) / 8));
    }
    if (bdp.bits) {
      const uint64_t* sx = host.data() + (node_bytes + lo_bytes) / 8;
      const uint32_t bits = bdp.bits;
      bdp = planb::bucket_dir_params(sx, sidx_n);
      if (bdp.bits != bits) return fail_detail(PLANB_EINVAL, "bucket directory size");
      planb::fill_bucket_dir(sx, sidx_n, bdp,
                             host.data() + (node_bytes + lo_bytes + sidx_bytes + dirb) / 8);
    }
    if (lidx_n) {
      uint64_t* lx = host.data() + lidx_off / 8;
      planb::fill_sidx(iv, t->L, t->L.D - 1, lx);
      const uint32_t bits = lbp.bits;
      lbp = planb::bucket_dir_params(lx, lidx_n, 2);
      if (lbp.bits != bits) return fail_detail(PLANB_EINVAL, "leaf bucket directory size");
      planb::fill_bucket_dir(lx, lidx_n, lbp, host.data() + (lidx_off + lidx_bytes) / 8);
    }
  }
  t->build_ms = ms_since(t0);

  auto t1 = std::chrono::steady_clock::now();
  DeviceGuard g(device);
  if (!g.ok) return PLANB_ECUDA;
  if (learned) {
    // bucket width of the index: keys under one level-s subtree (1 when it holds every key)
    uint64_t span = 1;
    if (s < t->L.D) {
      span = t->L.kl;
      for (uint32_t l = s; l + 1 < t->L.D; l++) span *= t->L.b;
    }
    const uint32_t iters = o.model_iters < 0 ? 2000u : static_cast<uint32_t>(o.model_iters);
    rc = planb::build_learned(iv, static_cast<uint32_t>(std::min<uint64_t>(span, 1u << 30)),
                              model_leaves, iters, 0.01f, 64u, t->model);
    if (rc) return rc;
  }
  t->bytes = lidx_off + lidx_bytes + lbdb + val_bytes + model_bytes;
  if (g_inject.load() == 2) {
    g_inject.store(0);
    return PLANB_ENOMEM;
  }
  if (cudaMalloc(&t->mem, t->bytes) != cudaSuccess) {
    t->mem = nullptr;
    cudaGetLastError();
    return PLANB_ENOMEM;
  }
  char* base = static_cast<char*>(t->mem);
  const size_t head = lidx_off + lidx_bytes + lbdb;
  t->dump_bytes = head + m * vw;
  if (on_dev) {
    // the index region's rounding tail is zero, as in the host-filled image
    const size_t sidx_used = static_cast<size_t>(sidx_n) * 16;
    if ((sidx_bytes > sidx_used &&
         cudaMemsetAsync(base + node_bytes + lo_bytes + sidx_used, 0, sidx_bytes - sidx_used,
                         bs->s) != cudaSuccess))
      return PLANB_ECUDA;
    rc = planb::gpu_fill(giv, t->L, format, s, sidx_n, base,
                         lo_bytes ? reinterpret_cast<uint64_t*>(base + node_bytes) : nullptr,
                         reinterpret_cast<uint64_t*>(base + node_bytes + lo_bytes),
                         base + head, bs->s);
    if (rc) return fail_detail(rc, "device layout fill", cudaGetLastError());
    if (lidx_n) {
      const size_t used = static_cast<size_t>(lidx_n) * 16;
      if (lidx_bytes > used &&
          cudaMemsetAsync(base + lidx_off + used, 0, lidx_bytes - used, bs->s) != cudaSuccess)
        return PLANB_ECUDA;
      rc = planb::gpu_fill_index(giv, t->L, t->L.D - 1, lidx_n,
                                 reinterpret_cast<uint64_t*>(base + lidx_off), bs->s);
      if (rc) return fail_detail(rc, "device leaf index fill", cudaGetLastError());
    }
    // The directories come from the indexes the device just wrote, filled on the device too; the
    // host reads only each index's first and last high halves, which size them.
    auto ends = [&](size_t off, uint64_t n, uint64_t& first, uint64_t& last) {
      return cudaMemcpyAsync(&first, base + off, 8, cudaMemcpyDeviceToHost, bs->s) ==
                 cudaSuccess &&
             cudaMemcpyAsync(&last, base + off + (n - 1) * 16, 8, cudaMemcpyDeviceToHost,
                             bs->s) == cudaSuccess &&
             cudaStreamSynchronize(bs->s) == cudaSuccess;
    };
    const size_t sidx_off = node_bytes + lo_bytes;
    if (dp.bits || bdp.bits) {
      uint64_t first = 0, last = 0;
      if (!ends(sidx_off, sidx_n, first, last))
        return fail_detail(PLANB_ECUDA, "device index ends", cudaGetLastError());
      const uint64_t* sx = reinterpret_cast<const uint64_t*>(base + sidx_off);
      if (dp.bits) {
        const uint32_t bits = dp.bits;
        dp = planb::dir_params_ends(first, last, sidx_n);
        if (dp.bits != bits) return fail_detail(PLANB_EINVAL, "radix directory size");
        if (cudaMemsetAsync(base + sidx_off + sidx_bytes, 0, dirb, bs->s) != cudaSuccess)
          return PLANB_ECUDA;
        rc = planb::gpu_fill_dir(sx, sidx_n, dp,
                                 reinterpret_cast<uint16_t*>(base + sidx_off + sidx_bytes), bs->s);
        if (rc) return fail_detail(rc, "device radix directory", cudaGetLastError());
      }
      if (bdp.bits) {
        const uint32_t bits = bdp.bits;
        bdp = planb::bucket_dir_params_ends(first, last, sidx_n);
        if (bdp.bits != bits) return fail_detail(PLANB_EINVAL, "bucket directory size");
        rc = planb::gpu_fill_bucket_dir(
            sx, sidx_n, bdp, reinterpret_cast<uint64_t*>(base + sidx_off + sidx_bytes + dirb),
            bs->s);
        if (rc) return fail_detail(rc, "device bucket directory", cudaGetLastError());
      }
    }
    if (lidx_n) {   // the leaf index's directory likewise
      uint64_t first = 0, last = 0;
      if (!ends(lidx_off, lidx_n, first, last))
        return fail_detail(PLANB_ECUDA, "device leaf index ends", cudaGetLastError());
      const uint32_t bits = lbp.bits;
      lbp = planb::bucket_dir_params_ends(first, last, lidx_n, 2);
      if (lbp.bits != bits) return fail_detail(PLANB_EINVAL, "leaf bucket directory size");
      rc = planb::gpu_fill_bucket_dir(reinterpret_cast<const uint64_t*>(base + lidx_off), lidx_n,
                                      lbp,
                                      reinterpret_cast<uint64_t*>(base + lidx_off + lidx_bytes),
                                      bs->s);
      if (rc) return fail_detail(rc, "device leaf bucket directory", cudaGetLastError());
    }
    if (cudaStreamSynchronize(bs->s) != cudaSuccess)
      return fail_detail(PLANB_ECUDA, "device directories", cudaGetLastError());
  } else {
    std::vector<uint32_t> words;
    const void* vals = iv.nh.data();
    if (format == PLANB_FMT_F16HI) {
      words.resize(m);
      planb::nh_words(iv, words.data());
      vals = words.data();
    }
    if (cudaMemcpy(base, host.data(), head, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + head, vals, m * vw, cudaMemcpyHostToDevice) != cudaSuccess)
      return PLANB_ECUDA;
  }
  if (learned) {
    char* mb = base + head + val_bytes;
    const size_t lb = static_cast<size_t>(model_leaves) * sizeof(planb::LeafModel);
    if (cudaMemcpy(mb, t->model.leaves.data(), lb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(mb + lb, t->model.err.data(), model_leaves * 2, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return PLANB_ECUDA;
    t->dt.leaves = reinterpret_cast<const planb::LeafModel*>(mb);
    t->dt.leaf_err = reinterpret_cast<const uint16_t*>(mb + lb);
    t->dt.lp = t->model.P;
  }
  t->dt.nodes = base;
  t->dt.nodes_lo = lo_bytes ? reinterpret_cast<const uint64_t*>(base + node_bytes) : nullptr;
  t->dt.sidx = sidx_n ? reinterpret_cast<const uint64_t*>(base + node_bytes + lo_bytes) : nullptr;
  t->dt.sidx_n = sidx_n;
  t->dt.sidx_node = s < t->L.D ? t->L.level_node[s] : 0;
  t->dt.dir = dp.bits ? reinterpret_cast<const uint16_t*>(base + node_bytes + lo_bytes + sidx_bytes)
                      : nullptr;
  t->dt.bdir = bdp.bits ? reinterpret_cast<const uint64_t*>(base + node_bytes + lo_bytes +
                                                          sidx_bytes + dirb)
                       : nullptr;
  t->dt.bdp = bdp;
  if (f16hyb && lidx_n) {
    t->dt.lidx = reinterpret_cast<const uint64_t*>(base + lidx_off);
    t->dt.lidx_n = lidx_n;
    t->dt.lidx_node = t->L.internal_nodes;   // the first leaf
    t->dt.lidx_db = 1;
    t->dt.lbdir = lbp.bits ? reinterpret_cast<const uint64_t*>(base + lidx_off + lidx_bytes)
                           : nullptr;
    t->dt.lbdp = lbp;
  } else if (f16hyb) {   // at most one level below the top-of-tree index: it serves
    t->dt.lidx = t->dt.sidx;
    t->dt.lidx_n = sidx_n;
    t->dt.lidx_node = t->dt.sidx_node;
    t->dt.lidx_db = t->L.D - s;
    t->dt.lbdir = t->dt.bdir;
    t->dt.lbdp = bdp;
  }
  t->dt.dir_bits = dp.bits;
  t->dt.dir_shift = dp.shift;
  t->dt.dir_base = dp.base;
  t->dt.kernel = kernel;
  t->dt.values = reinterpret_cast<const uint16_t*>(base + head);
  t->dt.n_intervals = m;
  t->dt.total_nodes = total;
  t->dt.internal_nodes = t->L.internal_nodes;
  t->dt.depth = t->L.D;
  t->dt.format = format;
  t->dt.smem_levels = s;
  t->dt.smem_nodes = kernel == planb::kCoop
                         ? static_cast<uint32_t>(planb::smem_bytes_for(t->L, format, s) / 128)
                         : 0;
  rc = planb::plan_launch(t->dt, device, o.block_threads, o.ctas_per_sm, t->cfg);
  if (rc) return rc;
  t->upload_ms = ms_since(t1);
  if (on_dev) {  // one device build: intervals, layout and fill together
    t->build_ms = ms_since(t0);
    t->upload_ms = 0;
  }
  out = std::move(t);
  return PLANB_OK;
}

// Frees retired tables whose grace period is over (see planb_update).
void reclaim(planb_fib* f, bool wait) {
  DeviceGuard g(f->device);
  for (auto it = f->retired.begin(); it != f->retired.end();) {
    Retired& r = *it;
    if (!r.fenced) {
      if (r.t.use_count() > 1 && !wait) { ++it; continue; }
      std::vector<cudaStream_t> ss;
      bool overflow;
      {
        std::lock_guard<std::mutex> lk(f->cur_mu);
        ss = f->streams;
        overflow = f->streams_overflow;
      }
      if (overflow || wait) {
        cudaDeviceSynchronize();
        r.events.clear();
      } else {
        for (cudaStream_t s : ss) {
          cudaEvent_t e;
          if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaDeviceSynchronize();
            break;
          }
          cudaEventRecord(e, s);
          r.events.push_back(e);
        }
      }
      r.fenced = true;
    }
    bool done = true;
    for (cudaEvent_t e : r.events) {
      cudaError_t q = wait ? cudaEventSynchronize(e) : cudaEventQuery(e);
      if (q == cudaErrorNotReady) { done = false; break; }
    }
    if (!done) { ++it; continue; }
    for (cudaEvent_t e : r.events) cudaEventDestroy(e);
    cudaGetLastError();
    it = f->retired.erase(it);
  }
}

void note_stream(planb_fib* f, cudaStream_t s) {
  for (cudaStream_t x : f->streams)
    if (x == s) return;
  if (f->streams.size() < 64) f->streams.push_back(s);
  else f->streams_overflow = true;
}

int canon_routes(const planb_route* r, size_t n, std::vector<planb::Prefix>& out) {
  std::vector<uint64_t> hi(n), lo(n);
  std::vector<uint8_t> len(n);
  std::vector<uint16_t> nh(n);
  for (size_t i = 0; i < n; i++) {
    hi[i] = r[i].hi; lo[i] = r[i].lo; len[i] = r[i].len; nh[i] = r[i].nexthop;
  }
  return planb::canonicalise(hi.data(), lo.data(), len.data(), nh.data(), n, out);
}

}  // namespace

extern "C" {

void planb_opts_default(planb_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(planb_opts);
  o->format = PLANB_FMT_F8X128;
  o->merge_equal_nh = 0;
  o->smem_levels = -1;
  o->device = -1;
  o->block_threads = 0;
  o->ctas_per_sm = 0;
  o->kernel = PLANB_KERNEL_AUTO;
  o->model_leaves = 0;
  o->model_iters = -1;
}

const char* planb_last_error(void) { return g_detail; }

const char* planb_strerror(int code) {
  switch (code) {
    case PLANB_OK: return "success";
    case PLANB_EINVAL: return "invalid argument";
    case PLANB_ENOMEM: return "out of memory";
    case PLANB_ECUDA: return "CUDA runtime error";
    case PLANB_EDEVICE: return "device-side check failed";
    case PLANB_ENODEV: return "no sm_103 CUDA device";
    case PLANB_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
  }
}

uint32_t planb_version(void) { return (1u << 16) | 0u; }

int planb_build(const uint64_t* prefix_hi, const uint64_t* prefix_lo, const uint8_t* len,
                const uint16_t* nexthop, size_t n, const planb_opts* opts, planb_fib** out) {
  if (!out) return PLANB_EINVAL;
  *out = nullptr;
  planb_opts o;
  planb_opts_default(&o);
  if (opts) {
    if (opts->struct_size < offsetof(planb_opts, reserved)) return PLANB_EINVAL;
    std::memcpy(&o, opts, std::min<size_t>(opts->struct_size, sizeof(o)));
    o.struct_size = sizeof(o);
  }
  if (o.format != PLANB_FMT_F8X128 && o.format != PLANB_FMT_F16HI && o.format != PLANB_FMT_F8V7)
    return PLANB_EINVAL;
  if (o.format == PLANB_FMT_F8V7 && o.kernel != PLANB_KERNEL_AUTO &&
      o.kernel != PLANB_KERNEL_HYBRID && o.kernel != PLANB_KERNEL_LEARNED)
    return PLANB_EINVAL;
  if (o.block_threads < 0 || o.block_threads > 512 || o.block_threads % 32) return PLANB_EINVAL;
  if (o.kernel < PLANB_KERNEL_AUTO || o.kernel > PLANB_KERNEL_LEARNED) return PLANB_EINVAL;
  if (o.format == PLANB_FMT_F16HI && o.kernel > PLANB_KERNEL_HYBRID) return PLANB_EINVAL;
  if (o.model_leaves < 0 || o.model_leaves > 8192 || o.model_iters < -1) return PLANB_EINVAL;
  if (o.builder != PLANB_BUILDER_HOST && o.builder != PLANB_BUILDER_DEVICE) return PLANB_EINVAL;
  try {
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return PLANB_ENODEV;
    int rc = check_device(dev);
    if (rc) return rc;
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<planb_fib> f(new planb_fib());
    f->opts = o;
    f->device = dev;
    DeviceGuard gdev(dev);  // declared first: outlives the stream and buffers below
    if (!gdev.ok) return PLANB_ECUDA;
    BuildStream bs;
    planb::DevBuf d_canon;  // device builder: the canonical list, made on the GPU
    if (o.builder == PLANB_BUILDER_DEVICE) {
      if (!bs.make()) return fail_detail(PLANB_ECUDA, "build stream");
      uint64_t N = 0;
      rc = planb::gpu_canonicalise(prefix_hi, prefix_lo, len, nexthop, n, bs.s, d_canon, N);
      if (rc) return fail_detail(rc, "device canonicalise", cudaGetLastError());
      f->rib.resize(N);
      if (N && cudaMemcpyAsync(f->rib.data(), d_canon.p, N * sizeof(planb::Prefix),
                               cudaMemcpyDeviceToHost, bs.s) != cudaSuccess)
        return PLANB_ECUDA;
      if (cudaStreamSynchronize(bs.s) != cudaSuccess) return PLANB_ECUDA;
    } else {
      rc = planb::canonicalise(prefix_hi, prefix_lo, len, nexthop, n, f->rib);
      if (rc) return rc;
    }
    double canon_ms = ms_since(t0);
    std::shared_ptr<Table> t;
    rc = make_table(f->rib, n, o, dev, t, o.builder == PLANB_BUILDER_DEVICE ? &bs : nullptr,
                    o.builder == PLANB_BUILDER_DEVICE ? &d_canon : nullptr);
    if (rc) return rc;
    t->build_ms += canon_ms;
    DeviceGuard g(dev);
    if (cudaMalloc(&f->d_status, sizeof(uint32_t)) != cudaSuccess) return PLANB_ENOMEM;
    if (cudaMemset(f->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return PLANB_ECUDA;
    f->cur = std::move(t);
    f->version = 1;
    *out = f.release();
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  } catch (...) {
    return PLANB_EINVAL;
  }
}

int planb_lookup(const planb_fib* fib_c, const uint64_t* d_addr_hi, const uint64_t* d_addr_lo,
                 size_t n, uint16_t* d_out, planb_stream_t stream) {
  if (!fib_c) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  if (!d_addr_hi || !d_addr_lo || !d_out) return PLANB_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_addr_hi) | reinterpret_cast<uintptr_t>(d_addr_lo)) & 7u ||
      reinterpret_cast<uintptr_t>(d_out) & 1u)
    return PLANB_EINVAL;
  planb_fib* f = const_cast<planb_fib*>(fib_c);
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk(f->cur_mu);
    t = f->cur;
    note_stream(f, reinterpret_cast<cudaStream_t>(stream));
  }
  DeviceGuard g(f->device);
  if (!g.ok) return PLANB_ECUDA;
  return planb::launch_lookup(t->dt, t->cfg, d_addr_hi, d_addr_lo, n, d_out, f->d_status, stream);
}

}  // extern "C"

namespace {
// The device addresses of page-locked host buffers (all of them, or false).
bool device_view(const void* const* host, void** dev, int k) {
  for (int i = 0; i < k; i++) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host[i]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    dev[i] = a.devicePointer;
  }
  return true;
}
}  // namespace

extern "C" {

int planb_lookup_mapped(const planb_fib* fib_c, const uint64_t* addr_hi, const uint64_t* addr_lo,
                        size_t n, uint16_t* out, planb_stream_t stream) {
  if (!fib_c) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  if (!addr_hi || !addr_lo || !out) return PLANB_EINVAL;
  if ((reinterpret_cast<uintptr_t>(addr_hi) | reinterpret_cast<uintptr_t>(addr_lo)) & 7u ||
      reinterpret_cast<uintptr_t>(out) & 1u)
    return PLANB_EINVAL;
  planb_fib* f = const_cast<planb_fib*>(fib_c);
  DeviceGuard g(f->device);
  if (!g.ok) return PLANB_ECUDA;
  // each buffer must be page-locked host memory the device can address (else no launch at all)
  const void* host[3] = {addr_hi, addr_lo, out};
  void* dev[3] = {nullptr, nullptr, nullptr};
  if (!device_view(host, dev, 3))
    return fail_detail(PLANB_EINVAL, "mapped lookup: not page-locked host memory");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk(f->cur_mu);
    t = f->cur;
    note_stream(f, st);
  }
  return planb::launch_lookup(t->dt, t->cfg, static_cast<const uint64_t*>(dev[0]),
                              static_cast<const uint64_t*>(dev[1]), n,
                              static_cast<uint16_t*>(dev[2]), f->d_status, st, nullptr, nullptr,
                              true);
}

int planb_lookup_host(planb_fib* f, const uint64_t* addr_hi, const uint64_t* addr_lo, size_t n,
                      uint16_t* out) {
  if (!f) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  if (!addr_hi || !addr_lo || !out) return PLANB_EINVAL;
  std::lock_guard<std::mutex> ul(f->upd_mu);
  DeviceGuard g(f->device);
  if (!g.ok) return PLANB_ECUDA;
  const size_t slot_bytes = kHostChunk * (8 + 8 + 2);
  if (!f->hbuf) {
    if (cudaMalloc(&f->hbuf, slot_bytes * kHostSlots) != cudaSuccess) {
      f->hbuf = nullptr;
      cudaGetLastError();
      return PLANB_ENOMEM;
    }
    for (int s = 0; s < kHostSlots; s++) {
      if (cudaStreamCreateWithFlags(&f->hs[s], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&f->he[s], cudaEventDisableTiming) != cudaSuccess)
        return PLANB_ECUDA;
    }
  }
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk(f->cur_mu);
    t = f->cur;
    for (int s = 0; s < kHostSlots; s++) note_stream(f, f->hs[s]);
  }
  // page-locked buffers: the kernel reads and writes them over the host link itself (no copies;
  // low halves only on a tie), which moves fewer bytes than the copy pipeline below
  {
    const void* host[3] = {addr_hi, addr_lo, out};
    void* dev[3] = {nullptr, nullptr, nullptr};
    if (!((reinterpret_cast<uintptr_t>(addr_hi) | reinterpret_cast<uintptr_t>(addr_lo)) & 7u) &&
        !(reinterpret_cast<uintptr_t>(out) & 1u) && device_view(host, dev, 3)) {
      int rc = planb::launch_lookup(t->dt, t->cfg, static_cast<const uint64_t*>(dev[0]),
                                    static_cast<const uint64_t*>(dev[1]), n,
                                    static_cast<uint16_t*>(dev[2]), f->d_status, f->hs[0],
                                    nullptr, nullptr, true);
      if (cudaStreamSynchronize(f->hs[0]) != cudaSuccess) rc = PLANB_ECUDA;
      return rc;
    }
  }
  int rc = PLANB_OK;
  size_t chunk_id = 0;
  for (size_t off = 0; off < n; off += kHostChunk, chunk_id++) {
    const size_t c = std::min(kHostChunk, n - off);
    const int s = static_cast<int>(chunk_id % kHostSlots);
    char* base = static_cast<char*>(f->hbuf) + slot_bytes * s;
    uint64_t* dh = reinterpret_cast<uint64_t*>(base);
    uint64_t* dl = dh + kHostChunk;
    uint16_t* dout = reinterpret_cast<uint16_t*>(dl + kHostChunk);
    cudaStream_t st = f->hs[s];
    if (cudaMemcpyAsync(dh, addr_hi + off, c * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dl, addr_lo + off, c * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = PLANB_ECUDA;
      break;
    }
    rc = planb::launch_lookup(t->dt, t->cfg, dh, dl, c, dout, f->d_status, st);
    if (rc) break;
    if (cudaMemcpyAsync(out + off, dout, c * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      rc = PLANB_ECUDA;
      break;
    }
  }
  for (int s = 0; s < kHostSlots; s++)
    if (cudaStreamSynchronize(f->hs[s]) != cudaSuccess) rc = PLANB_ECUDA;
  return rc;
}

int planb_update(planb_fib* f, const planb_route* inserts, size_t n_ins,
                 const planb_prefix* withdraws, size_t n_wd, planb_stream_t stream) {
  if (!f) return PLANB_EINVAL;
  if ((n_ins && !inserts) || (n_wd && !withdraws)) return PLANB_EINVAL;
  try {
    std::lock_guard<std::mutex> ul(f->upd_mu);
    auto t0 = std::chrono::steady_clock::now();
    // canonical batches
    std::vector<planb::Prefix> ins;
    int rc = canon_routes(inserts, n_ins, ins);
    if (rc) return rc;
    std::vector<planb::Prefix> wd(n_wd);
    for (size_t i = 0; i < n_wd; i++) {
      if (withdraws[i].len > 128) return PLANB_EINVAL;
      wd[i].p = planb::mk128(withdraws[i].hi, withdraws[i].lo) & planb::top_bits(withdraws[i].len);
      wd[i].len = withdraws[i].len;
      wd[i].nh = 0;
    }
    std::sort(wd.begin(), wd.end(), planb::prefix_less);
    // withdraws apply one after another: a repeat of a prefix in the same batch finds it gone
    const size_t n_wd_all = wd.size();
    wd.erase(std::unique(wd.begin(), wd.end(),
                         [](const planb::Prefix& a, const planb::Prefix& b) {
                           return a.p == b.p && a.len == b.len;
                         }),
             wd.end());
    uint64_t absent = n_wd_all - wd.size();
    // merge: rib minus withdraws, then union inserts (an insert of a present prefix modifies it)
    std::vector<planb::Prefix> mid;
    mid.reserve(f->rib.size());
    {
      size_t i = 0, j = 0;
      const auto& R = f->rib;
      while (i < R.size() || j < wd.size()) {
        if (j == wd.size() || (i < R.size() && planb::prefix_less(R[i], wd[j]))) {
          mid.push_back(R[i++]);
        } else if (i == R.size() || planb::prefix_less(wd[j], R[i])) {
          absent++;
          j++;
        } else {
          i++;
          j++;
        }
      }
    }
    std::vector<planb::Prefix> next;
    next.reserve(mid.size() + ins.size());
    {
      size_t i = 0, j = 0;
      while (i < mid.size() || j < ins.size()) {
        if (j == ins.size() || (i < mid.size() && planb::prefix_less(mid[i], ins[j]))) {
          next.push_back(mid[i++]);
        } else if (i == mid.size() || planb::prefix_less(ins[j], mid[i])) {
          next.push_back(ins[j++]);
        } else {
          next.push_back(ins[j++]);
          i++;
        }
      }
    }
    const double merge_ms = ms_since(t0);
    std::shared_ptr<Table> t;
    rc = make_table(next, next.size(), f->opts, f->device, t);
    if (rc) return rc;  // the current table is untouched
    t->build_ms += merge_ms;
    std::shared_ptr<Table> old;
    {
      std::lock_guard<std::mutex> lk(f->cur_mu);
      old = std::move(f->cur);
      f->cur = std::move(t);
      note_stream(f, reinterpret_cast<cudaStream_t>(stream));
    }
    f->rib.swap(next);
    f->version++;
    f->withdraw_absent += absent;
    f->retired.push_back(Retired{std::move(old), {}, false});
    reclaim(f, false);
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  } catch (...) {
    return PLANB_EINVAL;
  }
}

int planb_forget_stream(planb_fib* f, planb_stream_t stream) {
  if (!f) return PLANB_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DeviceGuard g(f->device);
  if (!g.ok) return PLANB_ECUDA;
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_detail(PLANB_ECUDA, "forget stream: synchronize", e);
  std::lock_guard<std::mutex> lk(f->cur_mu);
  f->streams.erase(std::remove(f->streams.begin(), f->streams.end(), s), f->streams.end());
  return PLANB_OK;
}

int planb_stats(const planb_fib* fib_c, planb_stats_t* out) {
  if (!fib_c || !out) return PLANB_EINVAL;
  planb_fib* f = const_cast<planb_fib*>(fib_c);
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk(f->cur_mu);
    t = f->cur;
  }
  std::memset(out, 0, sizeof(*out));
  out->n_input = t->n_input;
  out->n_prefixes = t->n_prefixes;
  out->n_intervals = t->dt.n_intervals;
  out->depth = t->L.D;
  out->keys_per_node = t->L.k;
  out->fanout = t->L.b;
  out->smem_levels = t->dt.smem_levels;
  out->format = t->dt.format;
  out->device = static_cast<uint32_t>(f->device);
  out->internal_nodes = t->L.internal_nodes;
  out->leaf_nodes = t->L.leaf_nodes;
  out->node_bytes = t->L.total_nodes() * 128 * (t->dt.format == PLANB_FMT_F16HI ? 2 : 1);
  out->value_bytes = t->dt.n_intervals * (t->dt.format == PLANB_FMT_F16HI ? 4 : 2);
  out->version = f->version;
  out->withdraw_absent = f->withdraw_absent;
  out->build_ms = t->build_ms;
  out->upload_ms = t->upload_ms;
  out->builder = t->builder;
  out->kernel = t->dt.kernel;
  out->threads = static_cast<uint32_t>(t->cfg.threads);
  out->ctas = static_cast<uint32_t>(t->cfg.blocks);
  out->smem_bytes = static_cast<uint32_t>(t->cfg.smem_bytes);
  if (t->dt.kernel == planb::kLearned) {
    out->model_leaves = t->model.P.leaves;
    out->model_iters = t->model.iters;
    out->model_max_err = t->model.max_err;
    out->model_loss0 = t->model.loss0;
    out->model_loss = t->model.loss;
    out->model_covered = t->model.covered;
    out->model_mean_err = t->model.mean_err;
    out->model_train_ms = t->model.train_ms;
  }
  return PLANB_OK;
}

int planb_device_status(planb_fib* f, uint32_t* detail) {
  if (!f) return PLANB_EINVAL;
  DeviceGuard g(f->device);
  if (!g.ok) return PLANB_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return PLANB_ECUDA;
  uint32_t w = 0;
  if (cudaMemcpy(&w, f->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PLANB_ECUDA;
  if (cudaMemset(f->d_status, 0, 4) != cudaSuccess) return PLANB_ECUDA;
  if (detail) *detail = w;
  if (w == 0) return PLANB_OK;
  return (w & 0x80000000u) ? PLANB_ETIMEOUT : PLANB_EDEVICE;
}

void planb_destroy(planb_fib* f) {
  if (!f) return;
  {
    std::lock_guard<std::mutex> ul(f->upd_mu);
    reclaim(f, true);
  }
  DeviceGuard g(f->device);
  cudaDeviceSynchronize();
  for (int s = 0; s < kHostSlots; s++) {
    if (f->hs[s]) cudaStreamDestroy(f->hs[s]);
    if (f->he[s]) cudaEventDestroy(f->he[s]);
  }
  if (f->hbuf) cudaFree(f->hbuf);
  if (f->d_status) cudaFree(f->d_status);
  f->cur.reset();
  delete f;
}

int planb_intervals(const uint64_t* prefix_hi, const uint64_t* prefix_lo, const uint8_t* len,
                    const uint16_t* nexthop, size_t n, int merge_equal_nh, uint64_t* out_start_hi,
                    uint64_t* out_start_lo, uint16_t* out_nh, size_t cap, size_t* out_m) {
  if (!out_m) return PLANB_EINVAL;
  try {
    std::vector<planb::Prefix> canon;
    int rc = planb::canonicalise(prefix_hi, prefix_lo, len, nexthop, n, canon);
    if (rc) return rc;
    planb::Intervals iv;
    planb::sweep(canon, merge_equal_nh != 0, iv);
    *out_m = iv.size();
    if (cap < iv.size() || !out_start_hi || !out_start_lo || !out_nh) return PLANB_EINVAL;
    for (size_t i = 0; i < iv.size(); i++) {
      out_start_hi[i] = planb::hi64(iv.start[i]);
      out_start_lo[i] = planb::lo64(iv.start[i]);
      out_nh[i] = iv.nh[i];
    }
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_intervals_device(const uint64_t* prefix_hi, const uint64_t* prefix_lo,
                           const uint8_t* len, const uint16_t* nexthop, size_t n,
                           int merge_equal_nh, uint64_t* out_start_hi, uint64_t* out_start_lo,
                           uint16_t* out_nh, size_t cap, size_t* out_m) {
  if (!out_m) return PLANB_EINVAL;
  try {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PLANB_ENODEV;
    int rc = check_device(dev);
    if (rc) return rc;
    BuildStream bs;
    if (!bs.make()) return PLANB_ECUDA;
    planb::DevBuf d_canon;
    planb::GpuIntervals giv;
    uint64_t N = 0;
    rc = planb::gpu_canonicalise(prefix_hi, prefix_lo, len, nexthop, n, bs.s, d_canon, N);
    if (rc) return fail_detail(rc, "device canonicalise", cudaGetLastError());
    rc = planb::gpu_sweep(d_canon.as<planb::Prefix>(), N, merge_equal_nh != 0, bs.s, giv);
    if (rc) return fail_detail(rc, "device interval sweep", cudaGetLastError());
    *out_m = giv.m;
    if (cap < giv.m || !out_start_hi || !out_start_lo || !out_nh) return PLANB_EINVAL;
    if (giv.m &&
        (cudaMemcpyAsync(out_start_hi, giv.hi.p, giv.m * 8, cudaMemcpyDeviceToHost, bs.s) !=
             cudaSuccess ||
         cudaMemcpyAsync(out_start_lo, giv.lo.p, giv.m * 8, cudaMemcpyDeviceToHost, bs.s) !=
             cudaSuccess ||
         cudaMemcpyAsync(out_nh, giv.nh.p, giv.m * 2, cudaMemcpyDeviceToHost, bs.s) !=
             cudaSuccess))
      return PLANB_ECUDA;
    return cudaStreamSynchronize(bs.s) == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_debug_table_dump(const planb_fib* fib_c, void* dst, size_t cap, size_t* out_bytes) {
  if (!fib_c || !out_bytes) return PLANB_EINVAL;
  planb_fib* f = const_cast<planb_fib*>(fib_c);
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk(f->cur_mu);
    t = f->cur;
  }
  *out_bytes = t->dump_bytes;
  if (!dst || cap < t->dump_bytes) return PLANB_EINVAL;
  DeviceGuard g(t->device);
  if (!g.ok) return PLANB_ECUDA;
  return cudaMemcpy(dst, t->mem, t->dump_bytes, cudaMemcpyDeviceToHost) == cudaSuccess
             ? PLANB_OK
             : PLANB_ECUDA;
}

int planb_layout_info(uint32_t keys_per_node, uint64_t n_keys, uint32_t depth_override,
                      planb_layout_t* out) {
  if (!out) return PLANB_EINVAL;
  planb::Layout L;
  int rc = planb::make_layout(keys_per_node, n_keys, depth_override, L);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  out->keys_per_node = L.k;
  out->fanout = L.b;
  out->depth = L.D;
  out->n_keys = n_keys;
  out->internal_nodes = L.internal_nodes;
  out->leaf_capacity = L.leaf_capacity;
  out->key_capacity = L.leaf_capacity * L.k;
  for (uint32_t l = 0; l < L.D && l < 16; l++) out->level_start[l] = L.level_node[l] * L.k;
  return PLANB_OK;
}

uint64_t planb_child_index(uint32_t keys_per_node, uint32_t d, uint64_t j, uint32_t c) {
  // in nodes: child c of node j on level d is node level_node(d+1) + j*b + c
  const uint64_t k = keys_per_node, b = k + 1;
  uint64_t level = 0, pw = 1;
  for (uint32_t l = 0; l <= d; l++) {
    level += pw;  // after the loop: level_node(d+1) = sum_{l<=d} b^l
    pw *= b;
  }
  return (level + j * b + c) * k;
}

int planb_mlp_grad(const float* d_u, const float* d_t, size_t n, const float* w, float* grad,
                   double* loss, planb_stream_t stream) {
  if ((n && (!d_u || !d_t)) || !w || !grad || !loss) return PLANB_EINVAL;
  try {
    return planb::mlp_grad_host(d_u, nullptr, d_t, n, w, grad, loss,
                                reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_mlp_grad_split(const float* d_u, const float* d_ulo, const float* d_t, size_t n,
                         const float* w, float* grad, double* loss, planb_stream_t stream) {
  if ((n && (!d_u || !d_ulo || !d_t)) || !w || !grad || !loss) return PLANB_EINVAL;
  try {
    return planb::mlp_grad_host(d_u, d_ulo, d_t, n, w, grad, loss,
                                reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_mlp_knot_step(const float* d_u, const float* d_ulo, const float* d_t, size_t n,
                        float* w, const float* knots, float* v, float* m, float* q, int32_t step,
                        float lr, double* loss, planb_stream_t stream) {
  if ((n && (!d_u || !d_t)) || !w || !knots || !v || !m || !q || !loss || step < 0)
    return PLANB_EINVAL;
  try {
    return planb::knot_step_host(d_u, d_ulo, d_t, n, w, knots, v, m, q, step, lr, loss,
                                 reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_mlp_forward(const float* d_u, size_t n, const float* w, float* d_y,
                      planb_stream_t stream) {
  if ((n && (!d_u || !d_y)) || !w) return PLANB_EINVAL;
  return planb::mlp_forward_host(d_u, n, w, d_y, reinterpret_cast<cudaStream_t>(stream));
}

int planb_debug_kernel_info(const planb_fib* f, int multi, int* out6) {
  if (!f || !out6) return PLANB_EINVAL;
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk(const_cast<planb_fib*>(f)->cur_mu);
    t = f->cur;
  }
  DeviceGuard g(f->device);
  int rc = planb::kernel_attributes(t->dt, multi != 0, out6);
  return rc ? rc : PLANB_OK;
}

int planb_debug_inject(int point) {
  if (point < 0 || point > 2) return PLANB_EINVAL;
  g_inject.store(point);
  return PLANB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------ multi-table lookups

struct planb_multi {
  int device = 0;
  std::vector<planb_fib*> fibs;  // not owned
  uint32_t T = 0;
  size_t cap = 0;
  uint32_t G = 0;                // bucketing chunks
  void* mem = nullptr;
  uint64_t *bhi = nullptr, *range = nullptr;
  uint32_t* bsrc = nullptr;       // input position of each bucketed address
  uint16_t* where = nullptr;      // each address's slot in its bucketing tile
  uint32_t* counts = nullptr;
  uint32_t* tile_start = nullptr; // per bucketing tile and table: run start in the bucketed arrays
  uint16_t* tile_base = nullptr;  // ... and its first slot in the tile
  uint16_t* bres = nullptr;      // results in bucketed order
  planb::MultiDesc* desc = nullptr;  // per-table descriptors of the single persistent launch
  planb::MultiDesc* hdesc = nullptr; // page-locked staging of the descriptors (stream-ordered copy)
  cudaEvent_t desc_copied = nullptr; // the last copy out of hdesc has been made
  bool persist = false;          // the current tables all fit the single persistent launch
  int persist_ctas = 0;
  size_t persist_smem = 0;
  bool direct_ok = false;        // the current tables can all take the direct launch
  bool direct = false;           // the direct launch is the form of the current graph
  uint64_t direct_hot = 0;       // bytes of table lines the direct launch keeps reading
  int direct_ctas = 0;
  bool g_direct = false;         // the form the captured graph was made with
  planb::DirectRec* drec = nullptr;     // per-table records of the direct launch
  planb::DirectRec* hdrec = nullptr;    // page-locked staging of the records
  cudaStream_t cap_stream = nullptr;
  static constexpr int kBranches = 4;          // per-table lookups run on this many streams
  cudaStream_t side[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  cudaGraphExec_t exec = nullptr;
  const void *g_hi = nullptr, *g_lo = nullptr, *g_tid = nullptr, *g_out = nullptr,
             *g_dn = nullptr;
  size_t g_n = 0;
  std::vector<std::shared_ptr<Table>> snap;  // the tables the captured graph reads
  std::mutex mu;
  uint32_t flags = 0;
  uint64_t captures = 0;         // graph captures so far
};

namespace {

// The multi-table pipeline on stream s: bucketing; the per-table lookups, which read and write
// disjoint segments; the gather. When captured (fork), the lookups are forked over the side
// streams and joined back on s: parallel branches of the graph, so one table's tail overlaps the
// next table's start, while the graph still runs on s alone. Direct launches stay on s (a table
// swap between forked launches would fence only s).
int multi_pipeline(planb_multi* m, const std::vector<std::shared_ptr<Table>>& cur,
                   const uint64_t* d_addr_hi, const uint64_t* d_addr_lo, const uint8_t* d_table,
                   size_t n, uint16_t* d_out, cudaStream_t s, const uint64_t* d_n, bool fork) {
  if (m->direct) {   // one launch, in input order: nothing to bucket or gather
    const int rc = planb::launch_multi_direct(m->drec, m->T, d_addr_hi, d_addr_lo, d_table, n,
                                              d_n, d_out, m->fibs[0]->d_status, m->direct_ctas,
                                              s);
    return rc ? fail_detail(rc, "multi: direct lookup", cudaGetLastError()) : PLANB_OK;
  }
  int rc = planb::launch_bucketing(d_addr_hi, d_table, n, m->T, m->G, m->counts, m->range,
                                   m->bhi, m->bsrc, m->where, m->tile_start, m->tile_base, s,
                                   d_n);
  if (rc) return fail_detail(rc, "multi: bucketing", cudaGetLastError());
  cudaError_t e = cudaSuccess;
  fork = fork && !m->persist;
  if (fork) {
    e = cudaEventRecord(m->fork, s);
    for (int k = 0; e == cudaSuccess && k < planb_multi::kBranches; k++)
      e = cudaStreamWaitEvent(m->side[k], m->fork, 0);
    if (e != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: fork", e);
  }
  if (m->persist) {
    rc = planb::launch_multi_persistent(
        m->desc, m->T, m->range, m->bhi, d_addr_lo, m->bsrc, m->bres,
        reinterpret_cast<unsigned long long*>(m->range + 2 * m->T + 3), m->fibs[0]->d_status,
        m->persist_ctas, m->persist_smem, s);
    if (rc) return fail_detail(rc, "multi: persistent lookup", cudaGetLastError());
  } else {
    for (uint32_t t = 0; t < m->T; t++) {
      rc = planb::launch_lookup(cur[t]->dt, cur[t]->cfg, m->bhi, d_addr_lo, n, m->bres,
                                m->fibs[t]->d_status,
                                fork ? m->side[t % planb_multi::kBranches] : s, m->range + t,
                                m->bsrc);
      if (rc) return fail_detail(rc, "multi: table lookup", cudaGetLastError());
    }
  }
  for (int k = 0; fork && e == cudaSuccess && k < planb_multi::kBranches; k++) {
    e = cudaEventRecord(m->join[k], m->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->join[k], 0);
  }
  if (e != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: join", e);
  rc = planb::launch_gather(m->where, m->tile_start, m->tile_base, m->bres, n, m->T, m->G, d_out,
                            s, d_n);
  if (rc) return fail_detail(rc, "multi: gather", cudaGetLastError());
  return PLANB_OK;
}

}  // namespace

extern "C" {

int planb_multi_create(planb_fib* const* fibs, uint32_t n_tables, size_t max_batch,
                       uint32_t flags, planb_multi** out) {
  if (!out) return PLANB_EINVAL;
  *out = nullptr;
  if (!fibs || n_tables == 0 || n_tables > 255 || max_batch == 0 ||
      max_batch >= (size_t(1) << 32))
    return PLANB_EINVAL;
  for (uint32_t t = 0; t < n_tables; t++) {
    if (!fibs[t] || fibs[t]->device != fibs[0]->device) return PLANB_EINVAL;
    std::lock_guard<std::mutex> lk(fibs[t]->cur_mu);
    const planb::DevTable& d = fibs[t]->cur->dt;
    if (d.kernel == planb::kLearned) return PLANB_EINVAL;   // no multi-table form
  }
  try {
    std::unique_ptr<planb_multi> m(new planb_multi());
    m->device = fibs[0]->device;
    m->fibs.assign(fibs, fibs + n_tables);
    m->T = n_tables;
    m->cap = max_batch;
    m->flags = flags;
    DeviceGuard g(m->device);
    if (!g.ok) return PLANB_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess)
      return PLANB_ECUDA;
    if (int rc = planb::bucketing_setup()) return rc;
    // bucketing chunks: eight per SM for large batches, but no more than one 2,048-address tile
    // each at max_batch, so a group sized for small batches (a serving slot) launches few blocks
    const size_t by_batch = (max_batch + 2047) / 2048;
    m->G = static_cast<uint32_t>(std::max<size_t>(1, std::min<size_t>(by_batch, size_t(sms) * 8u)));
    const size_t cap = max_batch;
    auto up = [](size_t x) { return ((x + 255) / 256) * 256; };
    const size_t tiles = planb::bucketing_tiles(cap, m->G) * (m->T + 1);
    const size_t where_off = up(cap * 12), bres_off = where_off + up(cap * 2),
                 counts_off = bres_off + up(cap * 2),
                 range_off = counts_off + up(static_cast<size_t>(m->T + 1) * m->G * 4);
    const size_t desc_off = range_off + up((2 * m->T + 4) * 8);
    const size_t tstart_off = desc_off + up(m->T * sizeof(planb::MultiDesc));
    const size_t tbase_off = tstart_off + up(tiles * 4);
    const size_t drec_off = tbase_off + up(tiles * 2);
    const size_t bytes = drec_off + up(m->T * sizeof(planb::DirectRec));
    if (cudaMalloc(&m->mem, bytes) != cudaSuccess) {
      m->mem = nullptr;
      cudaGetLastError();
      return PLANB_ENOMEM;
    }
    char* b = static_cast<char*>(m->mem);
    m->bhi = reinterpret_cast<uint64_t*>(b);
    m->bsrc = reinterpret_cast<uint32_t*>(b + up(cap * 8));
    m->where = reinterpret_cast<uint16_t*>(b + where_off);
    m->tile_start = reinterpret_cast<uint32_t*>(b + tstart_off);
    m->tile_base = reinterpret_cast<uint16_t*>(b + tbase_off);
    m->bres = reinterpret_cast<uint16_t*>(b + bres_off);
    m->counts = reinterpret_cast<uint32_t*>(b + counts_off);
    m->range = reinterpret_cast<uint64_t*>(b + range_off);
    m->desc = reinterpret_cast<planb::MultiDesc*>(b + desc_off);
    m->drec = reinterpret_cast<planb::DirectRec*>(b + drec_off);
    bool ok = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&m->desc_copied, cudaEventDisableTiming) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&m->hdesc),
                            m->T * sizeof(planb::MultiDesc), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&m->hdrec),
                            m->T * sizeof(planb::DirectRec), cudaHostAllocDefault) == cudaSuccess;
    for (int k = 0; ok && k < planb_multi::kBranches; k++)
      ok = cudaStreamCreateWithFlags(&m->side[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&m->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      planb_multi_destroy(m.release());
      return PLANB_ECUDA;
    }
    *out = m.release();
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

namespace {
int multi_lookup_impl(planb_multi* m, const uint64_t* d_addr_hi, const uint64_t* d_addr_lo,
                      const uint8_t* d_table, size_t n, uint16_t* d_out, planb_stream_t stream,
                      const uint64_t* d_n);
}

int planb_multi_lookup(planb_multi* m, const uint64_t* d_addr_hi, const uint64_t* d_addr_lo,
                       const uint8_t* d_table, size_t n, uint16_t* d_out, planb_stream_t stream) {
  return multi_lookup_impl(m, d_addr_hi, d_addr_lo, d_table, n, d_out, stream, nullptr);
}

int planb_multi_lookup_devn(planb_multi* m, const uint64_t* d_addr_hi, const uint64_t* d_addr_lo,
                            const uint8_t* d_table, const uint64_t* d_n, size_t max_n,
                            uint16_t* d_out, planb_stream_t stream) {
  if (!d_n) return PLANB_EINVAL;
  return multi_lookup_impl(m, d_addr_hi, d_addr_lo, d_table, max_n, d_out, stream, d_n);
}

}  // extern "C"

namespace {
// Decides whether the current tables can share the single persistent launch (every one a hybrid
// table) and writes their descriptors. An index (with its directory) of at most kSmemBudget bytes
// is staged in shared memory per CTA; a larger one (an F16HI table built for the single-table
// kernel's 224 KB) is searched in place, so that it does not cost every table resident CTAs.
// The descriptors are copied in stream order on st (from page-locked staging), so graphs already
// queued on st read the old ones and later ones the new, without a host-side wait.
int refresh_descriptors(planb_multi* m, const std::vector<std::shared_ptr<Table>>& cur,
                        cudaStream_t st) {
  m->persist = false;
  m->direct_ok = false;
  if (m->flags & PLANB_MULTI_PER_TABLE) return PLANB_OK;
  // the staging buffers are reused: their previous copy must have been made
  const cudaError_t ew = cudaEventSynchronize(m->desc_copied);
  if (ew != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: descriptor staging", ew);
  if (!(m->flags & PLANB_MULTI_BUCKETED)) {
    // The direct launch: every table F16HI hybrid with at most one level below its in-place
    // index, of fewer than 2^24 nodes (a node and its table share one 32-bit word in the group
    // hand-off) and 2^32 intervals.
    bool can = true;
    for (uint32_t t = 0; can && t < m->T; t++) {
      const planb::DevTable& d = cur[t]->dt;
      can = d.format == PLANB_FMT_F16HI && d.kernel == planb::kHybrid && d.lidx_db <= 1 &&
            (!d.lidx_n || d.lbdir) && d.total_nodes < (uint64_t(1) << 24) &&
            d.n_intervals <= (uint64_t(1) << 32);
    }
    int ctas = 0;
    if (can && planb::multi_direct_setup(m->device, m->T, &ctas) == PLANB_OK) {
      m->direct_hot = 0;
      for (uint32_t t = 0; t < m->T; t++) {
        const planb::DevTable& d = cur[t]->dt;
        // leaf high halves and next-hop words, 12 bytes per interval, the index and directory
        m->direct_hot += d.n_intervals * 12u + d.lidx_n * 16u +
                         (d.lbdir ? (uint64_t(16) << d.lbdp.bits) : 0u);
        planb::DirectRec& r = m->hdrec[t];
        r.idx = d.lidx_n ? d.lidx : nullptr;
        r.bdir = d.lidx_n ? d.lbdir : nullptr;
        r.bdir_base = d.lbdp.base;
        r.packed = d.lbdp.bits | (d.lbdp.shift << 8) | (d.lidx_db << 16);
        r.idx_node = static_cast<uint32_t>(d.lidx_node);
        r.nodes = static_cast<const uint64_t*>(d.nodes);
        r.words = reinterpret_cast<const uint32_t*>(d.values);
        r.nodes_lo = d.nodes_lo;
        r.nk = static_cast<uint32_t>(d.n_intervals - 1);
        r.internal_nodes = static_cast<uint32_t>(d.internal_nodes);
      }
      cudaError_t e = cudaMemcpyAsync(m->drec, m->hdrec, m->T * sizeof(planb::DirectRec),
                                      cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaEventRecord(m->desc_copied, st);
      if (e != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: direct records", e);
      m->direct_ok = true;
      m->direct_ctas = ctas;
    }
    cudaGetLastError();
  }
  planb::MultiDesc* hd = m->hdesc;
  uint64_t max_n = 0;
  for (uint32_t t = 0; t < m->T; t++) {
    const planb::DevTable& d = cur[t]->dt;
    if (d.kernel != planb::kHybrid || d.depth < d.smem_levels) return PLANB_OK;
    planb::MultiDesc& x = hd[t];
    x.nodes = d.nodes;
    x.sidx = d.sidx;
    x.values = d.values;
    x.sidx_n = static_cast<uint32_t>(d.sidx_n);
    x.sidx_node = static_cast<uint32_t>(d.sidx_node);
    x.internal_nodes = static_cast<uint32_t>(d.internal_nodes);
    x.db = d.depth - d.smem_levels;
    x.packed = d.format == PLANB_FMT_F8V7 ? 1u : 0u;
    x.n_intervals = d.n_intervals;
    x.dir = d.dir;
    x.dir_bits = d.dir_bits;
    x.dir_shift = d.dir_shift;
    x.dir_base = d.dir_base;
    x.f16 = d.format == PLANB_FMT_F16HI ? 1u : 0u;
    x.nodes_lo = d.nodes_lo;
    x.pad = 0;
    x.bdir = d.bdir;
    x.bdp = d.bdp;
    const uint64_t need = ((d.sidx_n + 1) & ~1ull) * 8u +
                          (d.dir_bits ? ((((1ull << d.dir_bits) + 1) + 7) & ~7ull) * 2u : 0u);
    x.staged = need <= kSmemBudget ? 1u : 0u;
    if (d.lidx && d.lidx_db == 1 && d.lidx != d.sidx) {
      // an F16HI index two or more levels above the leaves: search the leaf-level index in place
      // instead (one level below the search, so a group keeps all four addresses in flight)
      x.staged = 0;
      x.sidx = d.lidx;
      x.sidx_n = static_cast<uint32_t>(d.lidx_n);
      x.sidx_node = static_cast<uint32_t>(d.lidx_node);
      x.db = 1;
      x.dir = nullptr;
      x.dir_bits = 0;
      x.bdir = d.lbdir;
      x.bdp = d.lbdp;
    }
    if (x.staged) max_n = std::max<uint64_t>(max_n, need);
  }
  // rounded up to 16 KB, so that a table growing a little keeps the captured launch's size,
  // unless the rounding would cost resident CTAs
  const size_t exact = ((m->T + 3u) & ~1u) * 8u + max_n;
  size_t smem = exact;
  int ctas = 0, ctas_round = 0;
  if (planb::multi_persistent_setup(m->device, exact, &ctas) != PLANB_OK) {
    cudaGetLastError();
    return PLANB_OK;   // too large for one CTA: per-table launches
  }
  const size_t rounded = ((exact + 16383) / 16384) * 16384;
  if (planb::multi_persistent_setup(m->device, rounded, &ctas_round) == PLANB_OK &&
      ctas_round == ctas)
    smem = rounded;
  cudaGetLastError();
  cudaError_t e = cudaMemcpyAsync(m->desc, hd, m->T * sizeof(planb::MultiDesc),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(m->desc_copied, st);
  if (e != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: descriptors", e);
  m->persist = true;
  m->persist_ctas = ctas;
  m->persist_smem = smem;
  return PLANB_OK;
}

int multi_lookup_impl(planb_multi* m, const uint64_t* d_addr_hi, const uint64_t* d_addr_lo,
                      const uint8_t* d_table, size_t n, uint16_t* d_out, planb_stream_t stream,
                      const uint64_t* d_n) {
  if (!m) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  if (!d_addr_hi || !d_addr_lo || !d_table || !d_out || n > m->cap) return PLANB_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_addr_hi) | reinterpret_cast<uintptr_t>(d_addr_lo)) & 7u ||
      reinterpret_cast<uintptr_t>(d_out) & 1u)
    return PLANB_EINVAL;
  std::lock_guard<std::mutex> lk(m->mu);
  DeviceGuard g(m->device);
  if (!g.ok) return PLANB_ECUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<std::shared_ptr<Table>> cur(m->T);
  for (uint32_t t = 0; t < m->T; t++) {
    planb_fib* f = m->fibs[t];
    std::lock_guard<std::mutex> lk2(f->cur_mu);
    cur[t] = f->cur;
    note_stream(f, st);   // the graph runs on st; capture streams never execute work
  }
  bool changed = m->snap.size() != m->T;
  for (uint32_t t = 0; !changed && t < m->T; t++) changed = m->snap[t] != cur[t];
  // New tables: the persistent launch reads them through its descriptors, rewritten in stream
  // order, so its captured graph stays valid unless the launch's shape changed; per-table launches
  // carry the table pointers in their parameters and are captured again.
  bool reshape = false;
  if (changed) {
    const bool was = m->persist, was_direct = m->direct_ok;
    const int ctas = m->persist_ctas, dctas = m->direct_ctas;
    const size_t smem = m->persist_smem;
    int rc = refresh_descriptors(m, cur, st);
    if (rc) return rc;
    // per-table launches carry the tables in their parameters; the single launches read records
    // copied in stream order, unless the launch's own parameters changed
    reshape = (!m->persist && !m->direct_ok) || was != m->persist ||
              was_direct != m->direct_ok ||
              (m->persist && (ctas != m->persist_ctas || smem != m->persist_smem)) ||
              (m->direct_ok && dctas != m->direct_ctas);
  }
  // The direct form reads every table's lines at once: while they stay in L2 it beats grouping
  // the batch by table at every size; past that, only up to a batch size where the grouping's
  // passes cost more than the direct form's L2 misses (64 tables, 3.9 M prefixes, about 123 MB of
  // table lines: the direct form is ahead up to 2^24 addresses, the grouping from 2^25).
  constexpr uint64_t kDirectHotAll = uint64_t(32) << 20;
  constexpr size_t kDirectMaxBatch = size_t(1) << 24;
  m->direct = m->direct_ok && ((m->flags & PLANB_MULTI_DIRECT) || m->direct_hot <= kDirectHotAll ||
                               n <= kDirectMaxBatch || !m->persist);
  if (m->flags & PLANB_MULTI_NO_GRAPH) {
    if (changed) m->snap = cur;
    return multi_pipeline(m, cur, d_addr_hi, d_addr_lo, d_table, n, d_out, st, d_n, false);
  }
  const bool same = !reshape && m->exec && m->g_hi == d_addr_hi && m->g_lo == d_addr_lo &&
                    m->g_tid == d_table && m->g_out == d_out && m->g_n == n && m->g_dn == d_n &&
                    m->g_direct == m->direct;
  if (same && changed) m->snap = cur;   // the replayed graph reads the new descriptors
  if (!same) {
    // a table was swapped by an update, or the buffers changed: capture the pipeline again
    if (m->exec) {
      const cudaError_t es = cudaStreamSynchronize(st);
      if (es != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: wait for previous graph", es);
      cudaGraphExecDestroy(m->exec);
      m->exec = nullptr;
    }
    cudaGetLastError();   // start the capture with no stale launch error
    const cudaError_t eb = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (eb != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: begin capture", eb);
    const int rc =
        multi_pipeline(m, cur, d_addr_hi, d_addr_lo, d_table, n, d_out, m->cap_stream, d_n, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(m->cap_stream, &graph);
    if (rc != PLANB_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != PLANB_OK ? rc : fail_detail(PLANB_ECUDA, "multi: end capture", ec);
    }
    m->captures++;
    const cudaError_t ei = cudaGraphInstantiate(&m->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      m->exec = nullptr;
      return fail_detail(PLANB_ECUDA, "multi: instantiate graph", ei);
    }
    m->g_hi = d_addr_hi;
    m->g_lo = d_addr_lo;
    m->g_tid = d_table;
    m->g_out = d_out;
    m->g_n = n;
    m->g_dn = d_n;
    m->g_direct = m->direct;
    m->snap = cur;
  }
  const cudaError_t eg = cudaGraphLaunch(m->exec, st);
  if (eg != cudaSuccess) return fail_detail(PLANB_ECUDA, "multi: graph launch", eg);
  return PLANB_OK;
}
}  // namespace

extern "C" {

uint64_t planb_multi_captures(const planb_multi* m) {
  if (!m) return 0;
  std::lock_guard<std::mutex> lk(const_cast<planb_multi*>(m)->mu);
  return m->captures;
}

int planb_multi_persistent(const planb_multi* m) {
  if (!m) return PLANB_EINVAL;
  std::lock_guard<std::mutex> lk(const_cast<planb_multi*>(m)->mu);
  return (m->persist || m->direct) ? 1 : 0;
}

int planb_multi_mode(const planb_multi* m) {
  if (!m) return PLANB_EINVAL;
  std::lock_guard<std::mutex> lk(const_cast<planb_multi*>(m)->mu);
  return m->direct ? PLANB_MULTI_MODE_DIRECT
                   : (m->persist ? PLANB_MULTI_MODE_BUCKETED : PLANB_MULTI_MODE_PER_TABLE);
}

void planb_multi_destroy(planb_multi* m) {
  if (!m) return;
  {
    DeviceGuard g(m->device);
    cudaDeviceSynchronize();
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    for (int k = 0; k < planb_multi::kBranches; k++) {
      if (m->side[k]) cudaStreamDestroy(m->side[k]);
      if (m->join[k]) cudaEventDestroy(m->join[k]);
    }
    if (m->fork) cudaEventDestroy(m->fork);
    if (m->desc_copied) cudaEventDestroy(m->desc_copied);
    if (m->hdesc) cudaFreeHost(m->hdesc);
    if (m->hdrec) cudaFreeHost(m->hdrec);
    if (m->mem) cudaFree(m->mem);
  }
  delete m;
}

}  // extern "C"

// ------------------------------------------------------------ lookups without device allocation
//
// planb_lookup_host_noalloc stages addresses and results through one fixed device array declared
// below instead of buffers from cudaMalloc. The array lives in every GPU context that loads this
// library, for the life of the process. Its device address comes from cudaGetSymbolAddress, taken
// once per device on the first call with that device current (the array's name in host code is
// only a host-side stand-in). Calls share the array, so a process-wide lock serialises them, and
// each call waits for its own copies before it returns and releases the lock.
namespace {

constexpr size_t kNoAllocMaxKeys = PLANB_NOALLOC_MAX_KEYS;
constexpr size_t kNoAllocBytes = kNoAllocMaxKeys * (8 + 8 + 2);  // hi, lo, next hop: 4.5 MiB

__device__ __align__(256) unsigned char g_noalloc_stage[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};  // device address of g_noalloc_stage per device ordinal

// with g_noalloc_mu held and `dev` current
int noalloc_stage(int dev, void** out) {
  if (dev < 0 || dev >= 256) return PLANB_EINVAL;
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_stage) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return PLANB_ECUDA;
    }
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return PLANB_OK;
}

}  // namespace

extern "C" int planb_lookup_host_noalloc(const planb_fib* fib_c, const uint64_t* addr_hi,
                                         const uint64_t* addr_lo, size_t n, uint16_t* out,
                                         planb_stream_t stream) {
  if (!fib_c) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  if (!addr_hi || !addr_lo || !out) return PLANB_EINVAL;
  if (n > kNoAllocMaxKeys) return PLANB_EINVAL;
  planb_fib* f = const_cast<planb_fib*>(fib_c);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  DeviceGuard g(f->device);
  if (!g.ok) return PLANB_ECUDA;
  void* stage = nullptr;
  int rc = noalloc_stage(f->device, &stage);
  if (rc) return rc;
  std::shared_ptr<Table> t;
  {
    std::lock_guard<std::mutex> lk2(f->cur_mu);
    t = f->cur;
    note_stream(f, reinterpret_cast<cudaStream_t>(stream));
  }
  uint64_t* dh = static_cast<uint64_t*>(stage);
  uint64_t* dl = dh + kNoAllocMaxKeys;
  uint16_t* dout = reinterpret_cast<uint16_t*>(dl + kNoAllocMaxKeys);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // Once the first copy is queued, every return drains the stream first, so the lock is never
  // released while this call's copies or kernel may still touch the shared array.
  rc = PLANB_OK;
  if (cudaMemcpyAsync(dh, addr_hi, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dl, addr_lo, n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = PLANB_ECUDA;
  if (!rc) rc = planb::launch_lookup(t->dt, t->cfg, dh, dl, n, dout, f->d_status, stream);
  if (!rc && cudaMemcpyAsync(out, dout, n * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = PLANB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = PLANB_ECUDA;
  return rc;
}
