// Learned position model: device-side inference shared by the model-building kernels (learned.cu)
// and the lookup kernel (lookup.cu), so that the recorded error bounds are measured with exactly the
// arithmetic the lookups use.
//
// The model is a two-layer recursive model index over the table's keys (the inclusive interval
// ends), predicting for an address x the count of keys below x, i.e. its interval index:
//   root   u = (x.hi - kmin) / (kmax - kmin) (an integer range reduction, then a two-float
//          conversion), y = b2 + sum_h w2[h] * min(max(w1[h] * u + b1[h], 0), cap[h]) with 16
//          saturating ReLU units; leaf = floor(y * L) clamped to [0, L).
//   leaf   rank = a + s * (x.hi - base) in FP32, on the signed 64-bit distance to the leaf's base.
// Each leaf records the largest |predicted - true rank| over the keys routed to it, plus one for
// addresses between keys; a leaf whose bound exceeds the window limit is marked for the tree path.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "planb_internal.h"

namespace planb {

// The root's input is carried as an unevaluated sum u = uh + ul of two floats (about 48 bits), so
// that keys packed into a tiny part of the key range (a dense regional block) stay distinct; the
// first layer adds the parts in an order that keeps the sum exact near each knot.
// Saturating units keep every term of the output sum bounded by its unit's rise, so a steep segment
// (a dense block of keys) does not cost the rest of the curve its FP32 precision by cancellation.
__host__ __device__ __forceinline__ float mlp_eval(const MlpWeights& w, float uh, float ul) {
  float y = w.b2;
#pragma unroll
  for (int h = 0; h < kMlpHidden; h++) {
    const float z = fmaf(w.w1[h], ul, fmaf(w.w1[h], uh, w.b1[h]));
    y = fmaf(w.w2[h], fminf(fmaxf(z, 0.0f), w.cap[h]), y);
  }
  return y;
}

// (uh, ul) of (x - kmin) * inv_range for an offset d = x - kmin >= 0: uh = float(d) * inv_range
// rounded, ul = the rest (the conversion's and the product's rounding errors).
__host__ __device__ __forceinline__ void split_input(uint64_t d, float inv_range, float* uh,
                                                     float* ul) {
  const float f = static_cast<float>(d);                       // rounds to nearest
  const uint64_t fi = f >= 18446744073709551616.0f ? ~0ull : static_cast<uint64_t>(f);
  const long long r = static_cast<long long>(d - fi);          // |r| <= 2^39 for d < 2^64
  const float hi = f * inv_range;
  const float prod_err = fmaf(f, inv_range, -hi);              // exact error of the product
  *uh = hi;
  *ul = fmaf(static_cast<float>(r), inv_range, prod_err);
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t predict_leaf(const LearnedParams& P, uint64_t xh) {
  float uh, ul;
  split_input(xh > P.kmin ? xh - P.kmin : 0ull, P.inv_range, &uh, &ul);
  const float y = mlp_eval(P.mlp, uh, ul);
  int l = __float2int_rd(y * static_cast<float>(P.leaves));
  l = l < 0 ? 0 : l;
  return static_cast<uint32_t>(l) >= P.leaves ? P.leaves - 1u : static_cast<uint32_t>(l);
}

// predicted rank, clamped to [0, n_keys - 1]
__device__ __forceinline__ uint32_t predict_rank(const LearnedParams& P, const LeafModel& m,
                                                 uint64_t xh) {
  const float d = __ll2float_rn(static_cast<long long>(xh - m.base));
  const float r = fmaf(m.s, d, m.a);
  if (!(r > 0.0f)) return 0u;                                   // also catches NaN
  const float top = static_cast<float>(P.n_keys - 1u);
  return r >= top ? P.n_keys - 1u : static_cast<uint32_t>(__float2uint_rn(r));
}

// floor(v / span) for v < 2^24, through FP32 with a one-step correction
__device__ __forceinline__ uint32_t div_span(const LearnedParams& P, uint32_t v) {
  uint32_t q = static_cast<uint32_t>(static_cast<float>(v) * P.inv_span);
  if (q * P.span > v) q--;
  else if ((q + 1u) * P.span <= v) q++;
  return q;
}
#endif

// ---------------------------------------------------------------------------- host side

// A trained model: lookup parameters, the per-leaf models and error bounds, and build figures.
struct LearnedBuild {
  LearnedParams P{};
  std::vector<LeafModel> leaves;
  std::vector<uint16_t> err;   // per leaf: window half-width, or kLeafFallback
  double loss0 = 0, loss = 0;  // training loss before and after
  uint32_t iters = 0;
  uint32_t max_err = 0;        // largest bound over non-empty leaves (before the window limit)
  double covered = 0;          // fraction of keys in leaves within the window limit
  double mean_err = 0;         // mean bound over covered keys
  double train_ms = 0, build_ms = 0;
};

// Trains the root on the GPU (current device), fits the leaves and measures their error bounds.
// span: keys per index bucket; leaves: L; iters: Adam steps; max_window: largest bound kept.
int build_learned(const Intervals& iv, uint32_t span, uint32_t leaves, uint32_t iters, float lr,
                  uint32_t max_window, LearnedBuild& out);

// Full-batch gradient (and loss) of the root's mean squared error on device arrays u, t of n
// entries (input u + ulo when d_ulo is given), for weights w (host, 65 floats: w1, b1, w2, b2, cap);
// synchronous on `st`.
int mlp_grad_host(const float* d_u, const float* d_ulo, const float* d_t, size_t n,
                  const float* w_host, float* grad_host, double* loss_host, cudaStream_t st);

// One iteration of the training loop in knot-value form (the gradient kernel, then the knot-value
// Adam kernel) on host copies of the state: w (65) is read and rewritten (w2, b2 from the new knot
// values), v, m, q (17 each) are read and rewritten, c (17 knots) is read; `step` is the number of
// steps already taken. Synchronous on `st`.
int knot_step_host(const float* d_u, const float* d_ulo, const float* d_t, size_t n,
                   float* w_host, const float* c_host, float* v_host, float* m_host,
                   float* q_host, int32_t step, float lr, double* loss_host, cudaStream_t st);

// y = root(u) for device arrays; asynchronous on `st`.
int mlp_forward_host(const float* d_u, size_t n, const float* w_host, float* d_y, cudaStream_t st);

// (the forward entry point takes a single-float input: ul = 0)

}  // namespace planb
