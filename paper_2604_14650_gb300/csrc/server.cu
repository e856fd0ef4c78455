// Serving engine: continuous batching of lookup requests over many tables (VRFs), with route
// updates applied between batches and tables admitted against a device-memory budget.
//
// The paper's data plane turns NIC bursts into lookup batches and applies route changes by
// rebuild-and-swap on other cores (Sections 3.4, 3.6, 3.7). Here requests (one table, up to
// max_request addresses, host buffers) queue up; a dispatcher thread packs whatever is queued into
// the next free slot — a stream with pinned staging and device buffers of max_batch addresses — so
// requests that arrive while others run join the next batch instead of waiting for a fixed batch
// to fill, and several slots' copies and lookups overlap on the device. A slot's work is one
// multi-table pipeline (planb_multi_lookup_devn: the batch size is read from device memory, so the
// slot's captured graph is replayed for every batch). An updater thread applies queued route
// changes to their tables every update period (planb_update: rebuild and swap); batches formed
// after a swap see the new table.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "planb.h"

namespace {

using clock_t_ = std::chrono::steady_clock;

struct Request {
  uint32_t table = 0;
  const uint64_t* hi = nullptr;
  const uint64_t* lo = nullptr;
  size_t n = 0;
  uint16_t* out = nullptr;
  uint64_t ticket = 0;
  clock_t_::time_point t0;
  int status = 1;  // 1 = pending, PLANB_OK = done, < 0 = failed
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  uint64_t *h_hi = nullptr, *h_lo = nullptr, *h_n = nullptr;
  uint8_t* h_tid = nullptr;
  uint16_t* h_out = nullptr;
  void* dmem = nullptr;
  uint64_t *d_hi = nullptr, *d_lo = nullptr, *d_n = nullptr;
  uint8_t* d_tid = nullptr;
  uint16_t* d_out = nullptr;
  planb_multi* mt = nullptr;
  uint64_t tables_version = 0;  // table set the group was made for
  std::vector<std::shared_ptr<Request>> reqs;
  std::vector<size_t> offs;
  bool busy = false;
  std::chrono::steady_clock::time_point launched;
};

struct PendingUpdate {
  std::vector<planb_route> ins;
  std::vector<planb_prefix> wd;
};

}  // namespace

struct planb_server {
  planb_server_opts o{};
  int device = 0;
  std::mutex mu;                       // tables, queue, tickets, stats
  std::condition_variable cv_queue, cv_done;   // dispatcher wake-ups; request completions
  std::condition_variable cv_upd;              // the updater's period timer (and shutdown)
  std::vector<planb_fib*> tables;
  uint64_t tables_version = 0;
  uint64_t table_bytes = 0;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
  uint64_t next_ticket = 1;
  std::vector<Slot> slots;
  std::vector<PendingUpdate> pending;  // per table
  uint64_t pending_count = 0;
  std::atomic<bool> stop{false};
  std::thread dispatcher, updater;
  // statistics
  uint64_t requests = 0, lookups = 0, batches = 0, updates = 0, update_batches = 0;
  double rebuild_ms = 0;
  std::vector<float> lat_us;           // ring of recent request latencies
  size_t lat_pos = 0, lat_count = 0;
  std::vector<float> batch_us;         // ring of recent batch durations (launch to completion)
  size_t batch_pos = 0, batch_count = 0;
  int last_error = PLANB_OK;
  char last_detail[512] = "";
  uint64_t recaptures = 0;             // batches whose slot group saw a swapped table
};

namespace {

constexpr size_t kLatRing = size_t(1) << 20;
constexpr size_t kBatchRing = size_t(1) << 18;

// with m->mu held: remember a failure and where it happened
void note_error(planb_server* m, int rc, const char* where, const char* why) {
  m->last_error = rc;
  snprintf(m->last_detail, sizeof(m->last_detail), "%s: %s", where, why ? why : "");
}

void free_slot(Slot& s) {
  if (s.mt) planb_multi_destroy(s.mt);   // its captures are counted by the caller when it matters
  if (s.ev) cudaEventDestroy(s.ev);
  if (s.st) cudaStreamDestroy(s.st);
  if (s.h_hi) cudaFreeHost(s.h_hi);
  if (s.h_lo) cudaFreeHost(s.h_lo);
  if (s.h_tid) cudaFreeHost(s.h_tid);
  if (s.h_out) cudaFreeHost(s.h_out);
  if (s.h_n) cudaFreeHost(s.h_n);
  if (s.dmem) cudaFree(s.dmem);
  s = Slot();
}

int make_slot(Slot& s, size_t cap) {
  if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess)
    return PLANB_ECUDA;
  if (cudaHostAlloc(reinterpret_cast<void**>(&s.h_hi), cap * 8, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&s.h_lo), cap * 8, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&s.h_tid), cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&s.h_out), cap * 2, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&s.h_n), 8, cudaHostAllocDefault) != cudaSuccess)
    return PLANB_ENOMEM;
  const size_t bytes = cap * 16 + ((cap + 255) / 256) * 256 + ((cap * 2 + 255) / 256) * 256 + 256;
  if (cudaMalloc(&s.dmem, bytes) != cudaSuccess) return PLANB_ENOMEM;
  char* b = static_cast<char*>(s.dmem);
  s.d_hi = reinterpret_cast<uint64_t*>(b);
  s.d_lo = s.d_hi + cap;
  s.d_tid = reinterpret_cast<uint8_t*>(b + cap * 16);
  s.d_out = reinterpret_cast<uint16_t*>(b + cap * 16 + ((cap + 255) / 256) * 256);
  s.d_n = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(s.d_out) +
                                      ((cap * 2 + 255) / 256) * 256);
  return PLANB_OK;
}

// with m->mu held: results of a finished slot go to their requests
void complete_slot(planb_server* m, Slot& s, int status) {
  const auto now = clock_t_::now();
  if (!s.reqs.empty()) {
    m->batch_us[m->batch_pos] = std::chrono::duration<float, std::micro>(now - s.launched).count();
    m->batch_pos = (m->batch_pos + 1) % kBatchRing;
    m->batch_count++;
  }
  for (size_t i = 0; i < s.reqs.size(); i++) {
    Request& r = *s.reqs[i];
    if (status == PLANB_OK) std::memcpy(r.out, s.h_out + s.offs[i], r.n * 2);
    r.status = status;
    const float us = std::chrono::duration<float, std::micro>(now - r.t0).count();
    m->lat_us[m->lat_pos] = us;
    m->lat_pos = (m->lat_pos + 1) % kLatRing;
    m->lat_count++;
    m->requests++;
    m->lookups += r.n;
  }
  s.reqs.clear();
  s.offs.clear();
  s.busy = false;
  m->cv_done.notify_all();
}

// Runs on the CUDA runtime's callback thread when a slot's batch (copies, lookups, copies back)
// has finished: wakes the dispatcher at once instead of at its next poll. No CUDA calls here.
void CUDART_CB batch_done(void* user) {
  static_cast<planb_server*>(user)->cv_queue.notify_all();
}

void dispatcher_main(planb_server* m) {
  cudaSetDevice(m->device);
  size_t next_slot = 0;
  while (!m->stop.load()) {
    std::unique_lock<std::mutex> lk(m->mu);
    // finished slots first
    for (Slot& s : m->slots)
      if (s.busy && cudaEventQuery(s.ev) != cudaErrorNotReady) {
        const cudaError_t e = cudaEventSynchronize(s.ev);
        if (e != cudaSuccess) note_error(m, PLANB_ECUDA, "batch completion", cudaGetErrorString(e));
        complete_slot(m, s, e == cudaSuccess ? PLANB_OK : PLANB_ECUDA);
      }
    if (m->queue.empty()) {
      bool busy = false;
      for (Slot& s : m->slots) busy |= s.busy;
      // idle: sleep until work arrives; busy: until a batch finishes (its callback notifies),
      // with a short timeout as a fallback
      m->cv_queue.wait_for(lk, busy ? std::chrono::microseconds(200) : std::chrono::milliseconds(5));
      continue;
    }
    Slot* slot = nullptr;
    for (size_t k = 0; k < m->slots.size(); k++) {
      Slot& s = m->slots[(next_slot + k) % m->slots.size()];
      if (!s.busy) {
        slot = &s;
        next_slot = (next_slot + k + 1) % m->slots.size();
        break;
      }
    }
    if (!slot) {
      // every slot is in flight: wait for the oldest one outside the lock
      Slot& s = m->slots[next_slot];
      lk.unlock();
      cudaEventSynchronize(s.ev);
      continue;
    }
    // a group for the current table set
    if (!slot->mt || slot->tables_version != m->tables_version) {
      if (slot->mt) {
        m->recaptures += planb_multi_captures(slot->mt);
        planb_multi_destroy(slot->mt);
      }
      slot->mt = nullptr;
      const int rc = planb_multi_create(m->tables.data(), static_cast<uint32_t>(m->tables.size()),
                                        m->o.max_batch, m->o.multi_flags, &slot->mt);
      if (rc) {
        note_error(m, rc, "slot table group", planb_last_error());
        while (!m->queue.empty()) {
          m->queue.front()->status = rc;
          m->queue.pop_front();
        }
        m->cv_done.notify_all();
        continue;
      }
      slot->tables_version = m->tables_version;
    }
    // pack whatever is queued, up to max_batch addresses
    size_t total = 0;
    while (!m->queue.empty() && total + m->queue.front()->n <= m->o.max_batch) {
      std::shared_ptr<Request> r = m->queue.front();
      m->queue.pop_front();
      slot->reqs.push_back(r);
      slot->offs.push_back(total);
      total += r->n;
    }
    lk.unlock();
    for (size_t i = 0; i < slot->reqs.size(); i++) {
      const Request& r = *slot->reqs[i];
      std::memcpy(slot->h_hi + slot->offs[i], r.hi, r.n * 8);
      std::memcpy(slot->h_lo + slot->offs[i], r.lo, r.n * 8);
      std::memset(slot->h_tid + slot->offs[i], static_cast<int>(r.table), r.n);
    }
    *slot->h_n = total;
    slot->launched = clock_t_::now();
    cudaStream_t st = slot->st;
    bool ok =
        cudaMemcpyAsync(slot->d_n, slot->h_n, 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
        cudaMemcpyAsync(slot->d_hi, slot->h_hi, total * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
        cudaMemcpyAsync(slot->d_lo, slot->h_lo, total * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
        cudaMemcpyAsync(slot->d_tid, slot->h_tid, total, cudaMemcpyHostToDevice, st) == cudaSuccess;
    int rc = ok ? planb_multi_lookup_devn(slot->mt, slot->d_hi, slot->d_lo, slot->d_tid, slot->d_n,
                                          m->o.max_batch, slot->d_out,
                                          reinterpret_cast<planb_stream_t>(st))
                : PLANB_ECUDA;
    if (rc == PLANB_OK &&
        (cudaMemcpyAsync(slot->h_out, slot->d_out, total * 2, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaEventRecord(slot->ev, st) != cudaSuccess ||
         cudaLaunchHostFunc(st, batch_done, m) != cudaSuccess))
      rc = PLANB_ECUDA;
    const char* why = rc == PLANB_OK ? "" : (ok ? planb_last_error() : "staging copy");
    char why_copy[256];
    snprintf(why_copy, sizeof(why_copy), "%s", why);
    lk.lock();
    m->batches++;
    slot->busy = true;
    if (rc != PLANB_OK) {
      note_error(m, rc, "batch launch", why_copy);
      cudaStreamSynchronize(st);
      complete_slot(m, *slot, rc);
    }
  }
}

void updater_main(planb_server* m) {
  cudaSetDevice(m->device);
  while (!m->stop.load()) {
    std::vector<std::pair<uint32_t, PendingUpdate>> work;
    std::vector<planb_fib*> tabs;
    {
      std::unique_lock<std::mutex> lk(m->mu);
      m->cv_upd.wait_for(lk, std::chrono::microseconds(m->o.update_period_us));
      if (m->stop.load()) break;
      if (!m->pending_count) continue;
      for (uint32_t t = 0; t < m->pending.size(); t++) {
        PendingUpdate& p = m->pending[t];
        if (p.ins.empty() && p.wd.empty()) continue;
        work.emplace_back(t, std::move(p));
        p = PendingUpdate();
      }
      m->pending_count = 0;
      tabs = m->tables;
    }
    for (auto& w : work) {
      const auto t0 = clock_t_::now();
      const int rc = planb_update(tabs[w.first], w.second.ins.data(), w.second.ins.size(),
                                  w.second.wd.data(), w.second.wd.size(), nullptr);
      const double ms = std::chrono::duration<double, std::milli>(clock_t_::now() - t0).count();
      char why[256];
      snprintf(why, sizeof(why), "%s", rc ? planb_last_error() : "");
      std::lock_guard<std::mutex> lk(m->mu);
      if (rc) {
        note_error(m, rc, "route update", why);
      } else {
        m->updates += w.second.ins.size() + w.second.wd.size();
        m->update_batches++;
        m->rebuild_ms += ms;
      }
    }
  }
}

}  // namespace

extern "C" {

void planb_server_opts_default(planb_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(*o);
  o->slots = 4;
  o->max_batch = 1u << 18;
  o->max_request = 1u << 16;
  o->mem_budget = 0;
  o->update_period_us = 10000;
  o->device = -1;
}

int planb_server_create(const planb_server_opts* opts, planb_server** out) {
  if (!out) return PLANB_EINVAL;
  *out = nullptr;
  planb_server_opts o;
  planb_server_opts_default(&o);
  if (opts) {
    if (opts->struct_size < offsetof(planb_server_opts, reserved)) return PLANB_EINVAL;
    std::memcpy(&o, opts, std::min<size_t>(opts->struct_size, sizeof(o)));
    o.struct_size = sizeof(o);
  }
  if (o.slots < 1 || o.slots > 64 || o.max_batch < 1 || o.max_request < 1 ||
      o.max_request > o.max_batch || o.update_period_us < 100 ||
      (o.multi_flags & ~(PLANB_MULTI_NO_GRAPH | PLANB_MULTI_PER_TABLE | PLANB_MULTI_BUCKETED |
                          PLANB_MULTI_DIRECT)))
    return PLANB_EINVAL;
  try {
    std::unique_ptr<planb_server> m(new planb_server());
    m->o = o;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return PLANB_ENODEV;
    m->device = dev;
    if (cudaSetDevice(dev) != cudaSuccess) return PLANB_ENODEV;
    m->lat_us.assign(kLatRing, 0.0f);
    m->batch_us.assign(kBatchRing, 0.0f);
    m->slots.resize(o.slots);
    for (Slot& s : m->slots) {
      const int rc = make_slot(s, o.max_batch);
      if (rc) {
        for (Slot& x : m->slots) free_slot(x);
        return rc;
      }
    }
    planb_server* raw = m.release();
    raw->dispatcher = std::thread(dispatcher_main, raw);
    raw->updater = std::thread(updater_main, raw);
    *out = raw;
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_server_add_table(planb_server* m, planb_fib* fib, uint32_t* table_id) {
  if (!m || !fib || !table_id) return PLANB_EINVAL;
  planb_stats_t st;
  int rc = planb_stats(fib, &st);
  if (rc) return rc;
  if (st.device != static_cast<uint32_t>(m->device)) return PLANB_EINVAL;
  const uint64_t bytes = st.node_bytes + st.value_bytes;
  std::lock_guard<std::mutex> lk(m->mu);
  if (m->tables.size() >= 255) return PLANB_EINVAL;
  if (m->o.mem_budget && m->table_bytes + bytes > m->o.mem_budget) return PLANB_ENOMEM;
  m->table_bytes += bytes;
  *table_id = static_cast<uint32_t>(m->tables.size());
  m->tables.push_back(fib);
  m->pending.emplace_back();
  m->tables_version++;
  return PLANB_OK;
}

int planb_server_submit(planb_server* m, uint32_t table_id, const uint64_t* addr_hi,
                        const uint64_t* addr_lo, size_t n, uint16_t* out, uint64_t* ticket) {
  if (!m || !ticket) return PLANB_EINVAL;
  if (n == 0 || n > m->o.max_request || !addr_hi || !addr_lo || !out) return PLANB_EINVAL;
  try {
    auto r = std::make_shared<Request>();
    r->table = table_id;
    r->hi = addr_hi;
    r->lo = addr_lo;
    r->n = n;
    r->out = out;
    r->t0 = clock_t_::now();
    std::lock_guard<std::mutex> lk(m->mu);
    if (table_id >= m->tables.size()) return PLANB_EINVAL;
    r->ticket = m->next_ticket++;
    m->tickets[r->ticket] = r;
    m->queue.push_back(r);
    *ticket = r->ticket;
    m->cv_queue.notify_all();
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_server_wait(planb_server* m, uint64_t ticket, uint32_t timeout_us) {
  if (!m) return PLANB_EINVAL;
  std::unique_lock<std::mutex> lk(m->mu);
  auto it = m->tickets.find(ticket);
  if (it == m->tickets.end()) return PLANB_EINVAL;
  std::shared_ptr<Request> r = it->second;
  const auto deadline = clock_t_::now() + std::chrono::microseconds(timeout_us);
  while (r->status == 1) {
    if (m->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->status == 1)
      return PLANB_ETIMEOUT;
  }
  m->tickets.erase(ticket);
  return r->status;
}

int planb_server_update(planb_server* m, uint32_t table_id, const planb_route* inserts,
                        size_t n_ins, const planb_prefix* withdraws, size_t n_wd) {
  if (!m || (n_ins && !inserts) || (n_wd && !withdraws)) return PLANB_EINVAL;
  try {
    std::lock_guard<std::mutex> lk(m->mu);
    if (table_id >= m->tables.size()) return PLANB_EINVAL;
    PendingUpdate& p = m->pending[table_id];
    p.ins.insert(p.ins.end(), inserts, inserts + n_ins);
    p.wd.insert(p.wd.end(), withdraws, withdraws + n_wd);
    m->pending_count += n_ins + n_wd;
    return PLANB_OK;
  } catch (const std::bad_alloc&) {
    return PLANB_ENOMEM;
  }
}

int planb_server_stats(planb_server* m, planb_server_stats_t* out) {
  if (!m || !out) return PLANB_EINVAL;
  std::vector<float> lat, bat;
  uint64_t recaptures = 0;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    bat.assign(m->batch_us.begin(), m->batch_us.begin() + std::min(m->batch_count, kBatchRing));
    recaptures = m->recaptures;
    for (Slot& s : m->slots) recaptures += planb_multi_captures(s.mt);
    std::memset(out, 0, sizeof(*out));
    out->requests = m->requests;
    out->lookups = m->lookups;
    out->batches = m->batches;
    out->updates = m->updates;
    out->update_batches = m->update_batches;
    out->tables = m->tables.size();
    out->table_bytes = m->table_bytes;
    out->queued = m->queue.size();
    out->rebuild_ms_mean = m->update_batches ? m->rebuild_ms / m->update_batches : 0.0;
    out->mean_batch = m->batches ? static_cast<double>(m->lookups) / m->batches : 0.0;
    out->last_error = m->last_error;
    const size_t k = std::min(m->lat_count, kLatRing);
    lat.assign(m->lat_us.begin(), m->lat_us.begin() + k);
  }
  if (!lat.empty()) {
    auto pct = [&](double q) {
      const size_t i = std::min(lat.size() - 1, static_cast<size_t>(q * lat.size()));
      std::nth_element(lat.begin(), lat.begin() + i, lat.end());
      return static_cast<double>(lat[i]);
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = *std::max_element(lat.begin(), lat.end());
  }
  if (!bat.empty()) {
    auto pct = [&](double q) {
      const size_t i = std::min(bat.size() - 1, static_cast<size_t>(q * bat.size()));
      std::nth_element(bat.begin(), bat.begin() + i, bat.end());
      return static_cast<double>(bat[i]);
    };
    out->batch_p50_us = pct(0.50);
    out->batch_p99_us = pct(0.99);
    out->batch_max_us = *std::max_element(bat.begin(), bat.end());
  }
  out->recaptures = recaptures;
  return PLANB_OK;
}

int planb_server_error_detail(planb_server* m, char* buf, size_t cap) {
  if (!m || !buf || cap == 0) return PLANB_EINVAL;
  std::lock_guard<std::mutex> lk(m->mu);
  snprintf(buf, cap, "%s", m->last_detail);
  return PLANB_OK;
}

void planb_server_reset_stats(planb_server* m) {
  if (!m) return;
  std::lock_guard<std::mutex> lk(m->mu);
  m->requests = m->lookups = m->batches = m->updates = m->update_batches = 0;
  m->rebuild_ms = 0;
  m->lat_pos = m->lat_count = 0;
  m->batch_pos = m->batch_count = 0;
  m->recaptures = 0;
}

void planb_server_destroy(planb_server* m) {
  if (!m) return;
  m->stop.store(true);
  m->cv_queue.notify_all();
  m->cv_upd.notify_all();
  if (m->dispatcher.joinable()) m->dispatcher.join();
  if (m->updater.joinable()) m->updater.join();
  cudaSetDevice(m->device);
  for (Slot& s : m->slots) {
    if (s.st) {
      cudaStreamSynchronize(s.st);
      // the tables fence their updates on the streams they were used on: drop this one first
      for (planb_fib* f : m->tables) planb_forget_stream(f, reinterpret_cast<planb_stream_t>(s.st));
    }
    if (s.busy) {
      std::lock_guard<std::mutex> lk(m->mu);
      complete_slot(m, s, PLANB_OK);
    }
    free_slot(s);
  }
  {
    std::lock_guard<std::mutex> lk(m->mu);
    for (auto& r : m->queue) r->status = PLANB_EINVAL;
    m->cv_done.notify_all();
  }
  delete m;
}

}  // extern "C"
