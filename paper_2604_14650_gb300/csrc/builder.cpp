// Host builder of the linearized B+-tree (build steps a1-a4).
//
//   a1  canonicalise        Section 3.1 "Range Conversion": a prefix P/L covers [P, P + 2^(128-L)).
//   a2  events + sort       Section 3.1 "Interval Partitioning"; Algorithm 2 (Section 3.6) builds
//                           (address, next hop) events and sorts them.
//   a3  stack sweep         Algorithm 2's stack: at each boundary the top of the stack is the longest
//                           covering prefix, so its next hop belongs to the interval that starts there.
//   a4  layout              Section 3.2: internal levels in breadth-first order, then the leaves, in
//                           one flat array; every node full, padded with all-ones keys.
//
// Readings taken where the paper is loose:
//   * ranges use the exclusive end P + 2^(128-L) in 129-bit arithmetic; an end equal to 2^128 is not
//     a boundary (Algorithm 2 writes 2^(64-L), undefined for L > 64, and does not treat overflow);
//   * at one address, end events are applied before start events, and starts in ascending length, so
//     the longest prefix ends on top of the stack (Algorithm 2 names a (address, length) order but
//     its tuples carry no length);
//   * boundaries are de-duplicated: one interval per distinct boundary (Section 3.1's "at most 2N+1
//     intervals"), where Algorithm 2 would write one key per event;
//   * tree keys are the inclusive interval ENDS start[i+1] - 1 and the descent counts keys strictly
//     below the address, a true lower bound as Algorithm 1 states; the count is then exactly the
//     index of the interval holding the address. With start keys and a ">=" count (Listing 1), the
//     all-ones padding would tie with the address ffff:...:ffff.
#include <algorithm>
#include <cstring>
#include <thread>

#include "planb_internal.h"

namespace planb {

namespace {

// LSD radix sort of 128-bit keys with a 32-bit payload, 16-bit digits; skips digits that are
// constant over the input. Stable.
struct KeyIdx {
  u128 key;
  uint32_t idx;
  uint32_t pad;
};

void radix_sort(std::vector<KeyIdx>& a) {
  const size_t n = a.size();
  if (n < 2048) {
    std::stable_sort(a.begin(), a.end(),
                     [](const KeyIdx& x, const KeyIdx& y) { return x.key < y.key; });
    return;
  }
  std::vector<KeyIdx> tmp(n);
  std::vector<size_t> cnt(65536);
  for (int pass = 0; pass < 8; pass++) {
    const int shift = pass * 16;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (size_t i = 0; i < n; i++) cnt[static_cast<uint32_t>(a[i].key >> shift) & 0xFFFF]++;
    bool constant = false;
    for (size_t d = 0; d < 65536; d++) {
      if (cnt[d] == n) { constant = true; break; }
      if (cnt[d]) break;
    }
    if (constant) continue;
    size_t sum = 0;
    for (size_t d = 0; d < 65536; d++) {
      size_t c = cnt[d];
      cnt[d] = sum;
      sum += c;
    }
    for (size_t i = 0; i < n; i++) tmp[cnt[static_cast<uint32_t>(a[i].key >> shift) & 0xFFFF]++] = a[i];
    a.swap(tmp);
  }
}

}  // namespace

int canonicalise(const uint64_t* hi, const uint64_t* lo, const uint8_t* len, const uint16_t* nh,
                 size_t n, std::vector<Prefix>& out) {
  out.clear();
  if (n == 0) return PLANB_OK;
  if (!hi || !lo || !len || !nh) return PLANB_EINVAL;
  if (n >= (1ull << 32)) return PLANB_EINVAL;
  for (size_t i = 0; i < n; i++)
    if (len[i] > 128) return PLANB_EINVAL;
  // Sort key: masked prefix in the top 121 bits is not enough room for the length, so sort by
  // (prefix, len, input index) in two stable passes: by index order (input order is already the
  // index), then radix on the prefix after a stable bucket by length.
  std::vector<KeyIdx> ki(n);
  for (size_t i = 0; i < n; i++) {
    ki[i].key = mk128(hi[i], lo[i]) & top_bits(len[i]);
    ki[i].idx = static_cast<uint32_t>(i);
  }
  // stable bucket by length first (129 buckets), then a stable radix sort by prefix keeps
  // (prefix, len, index) order.
  {
    std::vector<size_t> cnt(130, 0);
    for (size_t i = 0; i < n; i++) cnt[len[ki[i].idx] + 1]++;
    for (int L = 0; L < 129; L++) cnt[L + 1] += cnt[L];
    std::vector<KeyIdx> tmp(n);
    for (size_t i = 0; i < n; i++) tmp[cnt[len[ki[i].idx]]++] = ki[i];
    ki.swap(tmp);
  }
  radix_sort(ki);
  out.reserve(n);
  for (size_t i = 0; i < n; i++) {
    const KeyIdx& e = ki[i];
    const uint8_t L = len[e.idx];
    // the last entry of each (prefix, len) run wins: it has the largest input index
    if (i + 1 < n && ki[i + 1].key == e.key && len[ki[i + 1].idx] == L) continue;
    out.push_back(Prefix{e.key, nh[e.idx], L});
  }
  return PLANB_OK;
}

void sweep(const std::vector<Prefix>& canon, bool merge_equal_nh, Intervals& out) {
  out.start.clear();
  out.nh.clear();
  const size_t S = canon.size();
  // end events: exclusive ends below 2^128 (a /0 and top-of-space prefixes have none)
  std::vector<KeyIdx> ends;
  ends.reserve(S);
  for (size_t i = 0; i < S; i++) {
    const Prefix& p = canon[i];
    if (p.len == 0) continue;
    const u128 width = static_cast<u128>(1) << (128 - p.len);
    const u128 e = p.p + width;  // wraps to 0 exactly when the end is 2^128
    if (e != 0) ends.push_back(KeyIdx{e, static_cast<uint32_t>(i), 0});
  }
  radix_sort(ends);
  out.start.reserve(S + ends.size() + 1);
  out.nh.reserve(S + ends.size() + 1);
  auto emit = [&](u128 a, uint16_t h) {
    if (merge_equal_nh && !out.nh.empty() && out.nh.back() == h) return;
    out.start.push_back(a);
    out.nh.push_back(h);
  };
  std::vector<uint16_t> stack;
  stack.reserve(130);
  size_t i = 0, j = 0;
  const size_t E = ends.size();
  const bool zero_is_event = (S > 0 && canon[0].p == 0);  // ends are never at 0
  if (!zero_is_event) emit(0, 0);
  while (i < S || j < E) {
    u128 a;
    if (i < S && j < E) a = std::min(canon[i].p, ends[j].key);
    else if (i < S) a = canon[i].p;
    else a = ends[j].key;
    while (j < E && ends[j].key == a) {  // the prefixes ending here are the top of the stack
      if (!stack.empty()) stack.pop_back();
      j++;
    }
    while (i < S && canon[i].p == a) {   // starts in ascending length: the longest ends on top
      stack.push_back(canon[i].nh);
      i++;
    }
    emit(a, stack.empty() ? static_cast<uint16_t>(0) : stack.back());
  }
}

int make_layout(uint32_t k, uint64_t n_keys, uint32_t depth_override, Layout& L, uint32_t kl) {
  if (k < 1) return PLANB_EINVAL;
  if (kl == 0) kl = k;
  if (kl > k) return PLANB_EINVAL;
  L = Layout();
  L.k = k;
  L.kl = kl;
  L.b = k + 1;
  L.n_keys = n_keys;
  uint32_t D = 1;
  if (depth_override) {
    D = depth_override;
  } else {
    u128 cap = kl;
    while (cap < n_keys) {
      cap *= L.b;
      D++;
      if (D > 16) return PLANB_EINVAL;
    }
  }
  if (D > 16) return PLANB_EINVAL;
  L.D = D;
  u128 acc = 0, pw = 1;
  for (uint32_t l = 0; l < D; l++) {
    L.level_node[l] = static_cast<uint64_t>(acc);
    if (l + 1 < D) acc += pw;
    pw *= L.b;
    if (pw > (static_cast<u128>(1) << 62)) return PLANB_EINVAL;
  }
  L.internal_nodes = static_cast<uint64_t>(acc);
  L.level_node[D] = L.internal_nodes;
  u128 lc = 1;
  for (uint32_t l = 0; l + 1 < D; l++) lc *= L.b;
  L.leaf_capacity = static_cast<uint64_t>(lc);
  // positions 0 .. n_keys must exist (the count can reach n_keys); leaves beyond are never visited
  const uint64_t need = (n_keys + 1 + kl - 1) / kl;
  L.leaf_nodes = std::min<uint64_t>(L.leaf_capacity, std::max<uint64_t>(need, 1));
  return PLANB_OK;
}

namespace {

// inclusive end of interval i (the tree key at leaf position i), or all-ones: for padding
// (pos >= n_keys) and for the last interval, which ends at 2^128 - 1
inline u128 key_at(const Intervals& iv, uint64_t n_keys, u128 pos) {
  if (pos >= n_keys || pos + 1 >= iv.size()) return ~static_cast<u128>(0);
  return iv.start[static_cast<size_t>(pos) + 1] - 1;
}

template <class Store>
void fill_generic(const Intervals& iv, const Layout& L, Store store) {
  const uint32_t k = L.k, kl = L.kl, b = L.b, D = L.D;
  // internal level l, node p, separator c: the largest key of child c's subtree, i.e. the key at
  // leaf position (p*b + c + 1) * b^(D-2-l) * kl - 1 (padding beyond the real keys)
  u128 span = 1;  // b^(D-2-l), leaves under one child of a level-l node
  for (uint32_t l = 0; l + 2 < D; l++) span *= b;
  for (uint32_t l = 0; l + 1 < D; l++) {
    const uint64_t nodes = L.level_node[l + 1] - L.level_node[l];
    for (uint64_t p = 0; p < nodes; p++) {
      const uint64_t node = L.level_node[l] + p;
      for (uint32_t c = 0; c < k; c++) {
        const u128 pos = (static_cast<u128>(p) * b + c + 1) * span * kl - 1;
        store(node, c, key_at(iv, L.n_keys, pos));
      }
    }
    span /= b;
  }
  auto leaf_range = [&](uint64_t j0, uint64_t j1) {
    for (uint64_t j = j0; j < j1; j++)
      for (uint32_t s = 0; s < kl; s++)
        store(L.internal_nodes + j, s, key_at(iv, L.n_keys, static_cast<u128>(j) * kl + s));
  };
  const uint64_t leaves = L.leaf_nodes;
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (leaves < 65536 || hw == 1) {
    leaf_range(0, leaves);
  } else {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < hw; t++)
      th.emplace_back(leaf_range, leaves * t / hw, leaves * (t + 1) / hw);
    for (auto& x : th) x.join();
  }
}

}  // namespace

void fill_f8x128(const Intervals& iv, const Layout& L, uint64_t* nodes) {
  fill_generic(iv, L, [nodes, k = L.k](uint64_t node, uint32_t slot, u128 key) {
    nodes[(node * k + slot) * 2 + 0] = hi64(key);
    nodes[(node * k + slot) * 2 + 1] = lo64(key);
  });
}

void fill_f8v7(const Intervals& iv, const Layout& L, uint64_t* nodes) {
  fill_generic(iv, L, [nodes, k = L.k](uint64_t node, uint32_t slot, u128 key) {
    nodes[(node * k + slot) * 2 + 0] = hi64(key);
    nodes[(node * k + slot) * 2 + 1] = lo64(key);
  });
  // slot 7 of every leaf: the next hops of its 7 keys
  const uint32_t kl = L.kl;
  for (uint64_t j = 0; j < L.leaf_nodes; j++) {
    uint64_t w[2] = {0, 0};
    for (uint32_t s = 0; s < kl; s++) {
      const uint64_t pos = j * kl + s;
      const uint64_t h = pos < iv.size() ? iv.nh[pos] : 0;
      w[s / 4] |= h << (16 * (s % 4));
    }
    const uint64_t node = L.internal_nodes + j;
    nodes[(node * L.k + kl) * 2 + 0] = w[0];
    nodes[(node * L.k + kl) * 2 + 1] = w[1];
  }
}

void nh_words(const Intervals& iv, uint32_t* out) {
  const uint64_t m = iv.nh.size();
  for (uint64_t i = 0; i < m; i++)
    out[i] = iv.nh[i] | ((i + 1 < m && lo64(iv.start[i + 1]) != 0) ? (1u << 16) : 0u);
}

void fill_f16hi(const Intervals& iv, const Layout& L, uint64_t* node_hi, uint64_t* node_lo) {
  fill_generic(iv, L, [node_hi, node_lo, k = L.k](uint64_t node, uint32_t slot, u128 key) {
    node_hi[node * k + slot] = hi64(key);
    node_lo[node * k + slot] = lo64(key);
  });
}

uint64_t sidx_entries(const Layout& L, uint32_t S) {
  if (S >= L.D) return L.n_keys;
  u128 span = L.kl;                    // keys under one level-S node: kl * b^(D-1-S)
  for (uint32_t l = S; l + 1 < L.D; l++) span *= L.b;
  u128 cap = 1;
  for (uint32_t l = 0; l < S; l++) cap *= L.b;
  const u128 full = static_cast<u128>(L.n_keys) / span;  // entries (q+1)*span-1 < n_keys
  return static_cast<uint64_t>(std::min<u128>(cap - 1, full));
}

void fill_sidx(const Intervals& iv, const Layout& L, uint32_t S, uint64_t* out) {
  const uint64_t n = sidx_entries(L, S);
  u128 span = 1;
  if (S < L.D) {
    span = L.kl;
    for (uint32_t l = S; l + 1 < L.D; l++) span *= L.b;
  }
  for (uint64_t q = 0; q < n; q++) {
    const u128 key = key_at(iv, L.n_keys, (static_cast<u128>(q) + 1) * span - 1);
    out[2 * q] = hi64(key);
    out[2 * q + 1] = lo64(key);
  }
}

uint32_t dir_bits_for(uint64_t n) {
  if (n == 0 || n >= 65536) return 0;
  uint32_t lg = 0;
  while ((uint64_t(1) << lg) < n) lg++;
  return std::min<uint32_t>(13, std::max<uint32_t>(4, lg + 1));   // about two buckets per entry
}

DirParams dir_params_ends(uint64_t lo, uint64_t hi, uint64_t n) {
  DirParams p;
  p.bits = dir_bits_for(n);
  if (!p.bits) return p;
  const uint64_t cap = uint64_t(1) << p.bits;
  while (p.shift < 63 && (hi >> p.shift) - (lo >> p.shift) >= cap) p.shift++;
  p.base = lo >> p.shift;
  return p;
}

DirParams dir_params(const uint64_t* sidx, uint64_t n) {
  return n ? dir_params_ends(sidx[0], sidx[2 * (n - 1)], n) : DirParams{};
}

void fill_dir(const uint64_t* sidx, uint64_t n, const DirParams& p, uint16_t* dir) {
  const uint64_t buckets = uint64_t(1) << p.bits;
  uint64_t q = 0;
  for (uint64_t b = 0; b <= buckets; b++) {
    while (q < n && (sidx[2 * q] >> p.shift) - p.base < b) q++;
    dir[b] = static_cast<uint16_t>(q);
  }
}

uint32_t bucket_dir_bits_for(uint64_t n, uint32_t extra) {
  if (n == 0 || n >= (uint64_t(1) << 31)) return 0;
  uint32_t lg = 0;
  while ((uint64_t(1) << lg) < n) lg++;
  return std::min<uint32_t>(20, std::max<uint32_t>(4, lg + extra));   // 2^extra buckets per entry
}

BucketDir bucket_dir_params_ends(uint64_t lo, uint64_t hi, uint64_t n, uint32_t extra) {
  BucketDir p;
  p.bits = bucket_dir_bits_for(n, extra);
  if (!p.bits) return p;
  const uint64_t cap = uint64_t(1) << p.bits;
  while (p.shift < 63 && (hi >> p.shift) - (lo >> p.shift) >= cap) p.shift++;
  p.base = lo >> p.shift;
  return p;
}

BucketDir bucket_dir_params(const uint64_t* sidx, uint64_t n, uint32_t extra) {
  return n ? bucket_dir_params_ends(sidx[0], sidx[2 * (n - 1)], n, extra) : BucketDir{};
}

void fill_bucket_dir(const uint64_t* sidx, uint64_t n, const BucketDir& p, uint64_t* out) {
  const uint64_t buckets = uint64_t(1) << p.bits;
  uint64_t q = 0;
  for (uint64_t b = 0; b < buckets; b++) {
    const uint64_t first = q;
    while (q < n && (sidx[2 * q] >> p.shift) - p.base <= b) q++;   // the entries of bucket b
    out[2 * b] = first | ((q - first) << 32);
    out[2 * b + 1] = first < n ? sidx[2 * first] : ~0ull;
  }
}

}  // namespace planb
