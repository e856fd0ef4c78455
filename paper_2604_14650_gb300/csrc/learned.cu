// Learned position model (the root MLP of a two-layer recursive model index): training on the GPU
// by hand-written forward/backward and Adam kernels, leaf fitting, and the error bounds the lookup
// kernel relies on. Inference arithmetic lives in learned.cuh and is shared with lookup.cu.
//
// Training fits the root to the empirical CDF of the keys: targets t_i = (i + 0.5) / n for the i-th
// key's range-reduced high half u_i, loss L = mean (y(u_i) - t_i)^2, full batch. The gradient
// kernel accumulates per-thread sums, reduces them per block in a fixed order and writes one row
// of 50 partials (49 gradients + the loss) per block; the update kernel adds the rows in block
// order in double precision and applies Adam (Kingma and Ba, 2015). The result is deterministic for
// a given grid. The iterations are captured once in a CUDA graph and replayed.
//
// Training starts from the piecewise-linear interpolation of the CDF through the inputs' 16
// quantiles (the hidden units' knots, kept fixed) and fits the output layer — a convex least-squares
// problem for fixed knots — by Adam on the spline's values at the knots (knot_adam_kernel). Without
// training the root is the identity (plain linear range reduction).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "learned.cuh"
#include "planb_internal.h"

namespace planb {

namespace {

constexpr int kRow = kMlpParams + 1;     // 49 gradients + loss
constexpr int kGradThreads = 256;
constexpr int kGradBlocks = 304;         // fixed grid: the partial sums' order never changes

__global__ void __launch_bounds__(kGradThreads) mlp_grad_kernel(const float* __restrict__ u,
                                                                const float* __restrict__ ulo,
                                                                const float* __restrict__ t,
                                                                uint32_t n,
                                                                const float* __restrict__ w,
                                                                float* __restrict__ partials) {
  __shared__ float sw[kMlpWeights];
  __shared__ float red[kGradThreads / 32][kRow];
  if (threadIdx.x < kMlpWeights) sw[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  float g[kRow];
#pragma unroll
  for (int k = 0; k < kRow; k++) g[k] = 0.0f;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float ui = u[i];
    const float li = ulo ? ulo[i] : 0.0f;
    float z[kMlpHidden];
    float y = sw[3 * kMlpHidden];
#pragma unroll
    for (int h = 0; h < kMlpHidden; h++) {
      z[h] = fmaf(sw[h], li, fmaf(sw[h], ui, sw[kMlpHidden + h]));
      y = fmaf(sw[2 * kMlpHidden + h], fminf(fmaxf(z[h], 0.0f), sw[kMlpParams + h]), y);
    }
    const float r = y - t[i];
    const float dy = 2.0f * r;              // the 1/n of the mean is applied after the reduction
    g[3 * kMlpHidden] += dy;
    g[kMlpParams] = fmaf(r, r, g[kMlpParams]);
#pragma unroll
    for (int h = 0; h < kMlpHidden; h++) {
      const float cap = sw[kMlpParams + h];
      const bool on = z[h] > 0.0f && z[h] < cap;          // the unit's slope is 1 inside (0, cap)
      g[2 * kMlpHidden + h] = fmaf(dy, fminf(fmaxf(z[h], 0.0f), cap), g[2 * kMlpHidden + h]);
      const float dz = on ? dy * sw[2 * kMlpHidden + h] : 0.0f;
      g[h] = fmaf(dz, ui + li, g[h]);
      g[kMlpHidden + h] += dz;
    }
  }
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRow; k++) {
    float v = g[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kRow) {
    float s = 0.0f;
    for (int wi = 0; wi < kGradThreads / 32; wi++) s += red[wi][threadIdx.x];
    partials[blockIdx.x * kRow + threadIdx.x] = s;
  }
}

// Sums the partial rows (block order, double) into grad[49] and loss (no update). Used for the
// loss before and after training and by planb_mlp_grad.
__global__ void reduce_kernel(const float* __restrict__ partials, uint32_t nblocks, uint32_t n,
                              float* __restrict__ grad_out, double* __restrict__ loss_out) {
  const int k = threadIdx.x;
  if (k >= kRow) return;
  double s = 0.0;
  for (uint32_t b = 0; b < nblocks; b++) s += static_cast<double>(partials[b * kRow + k]);
  const double mean = n ? s / static_cast<double>(n) : 0.0;
  if (k == kMlpParams) {
    if (loss_out) *loss_out = mean;
  } else if (grad_out) {
    grad_out[k] = static_cast<float>(mean);
  }
}

// One training step on the piecewise-linear root in knot-value form. With unit input weights,
// fixed knots c_0 < .. < c_16 (c_h = -b1[h], c_16 the largest input) and caps c_{h+1} - c_h, the
// network is the linear spline through (c_h, v_h): b2 = v_0 and w2[h] = s_h = (v_{h+1} - v_h) /
// (c_{h+1} - c_h). Adam (Kingma and Ba, 2015) runs on v, which is well conditioned (CDF values in
// [0, 1]); dL/dv comes from the network's gradient by the chain rule through those relations:
//   dL/dv_j = dL/dw2[j-1] / (c_j - c_{j-1}) - dL/dw2[j] / (c_{j+1} - c_j) (+ dL/db2 for j = 0).
// The new v is written back as (w2, b2). State: v[17], m[17], q[17] (moments), knots c[17].
__global__ void knot_adam_kernel(const float* __restrict__ partials, uint32_t nblocks, uint32_t n,
                                 float* __restrict__ w, float* __restrict__ v,
                                 float* __restrict__ m, float* __restrict__ q,
                                 const float* __restrict__ c, int* __restrict__ step, float lr,
                                 double* __restrict__ loss_out) {
  __shared__ float g[kRow];
  __shared__ float vs[kMlpHidden + 1];
  const int k = threadIdx.x;
  if (k < kRow) {
    double s = 0.0;
    for (uint32_t b = 0; b < nblocks; b++) s += static_cast<double>(partials[b * kRow + k]);
    const double mean = n ? s / static_cast<double>(n) : 0.0;
    g[k] = static_cast<float>(mean);
    if (k == kMlpParams && loss_out) *loss_out = mean;
  }
  __syncthreads();
  if (k <= kMlpHidden) {
    float gv = 0.0f;
    if (k >= 1) gv += g[2 * kMlpHidden + k - 1] / (c[k] - c[k - 1]);
    if (k < kMlpHidden) gv -= g[2 * kMlpHidden + k] / (c[k + 1] - c[k]);
    if (k == 0) gv += g[3 * kMlpHidden];
    const int tstep = *step + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mk = b1 * m[k] + (1.0f - b1) * gv;
    const float qk = b2 * q[k] + (1.0f - b2) * gv * gv;
    m[k] = mk;
    q[k] = qk;
    const float mh = mk / (1.0f - powf(b1, static_cast<float>(tstep)));
    const float qh = qk / (1.0f - powf(b2, static_cast<float>(tstep)));
    const float nv = v[k] - lr * mh / (sqrtf(qh) + eps);
    v[k] = nv;
    vs[k] = nv;
  }
  __syncthreads();
  if (k < kMlpHidden) w[2 * kMlpHidden + k] = (vs[k + 1] - vs[k]) / (c[k + 1] - c[k]);
  if (k == 0) w[3 * kMlpHidden] = vs[0];
}

__global__ void bump_step(int* step) { *step += 1; }

__global__ void mlp_forward_kernel(const float* __restrict__ u, uint32_t n, MlpWeights w,
                                   float* __restrict__ y) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = mlp_eval(w, u[i], 0.0f);
}

__global__ void leaf_assign_kernel(const uint64_t* __restrict__ khi, uint32_t n, LearnedParams P,
                                   uint32_t* __restrict__ leaf) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    leaf[i] = predict_leaf(P, khi[i]);
}

__global__ void leaf_error_kernel(const uint64_t* __restrict__ khi, uint32_t n, LearnedParams P,
                                  const LeafModel* __restrict__ leaves,
                                  uint32_t* __restrict__ err) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t l = predict_leaf(P, khi[i]);
    const uint32_t p = predict_rank(P, leaves[l], khi[i]);
    const uint32_t e = p > i ? p - i : i - p;
    atomicMax(err + l, e);
  }
}

void init_weights(MlpWeights& w) {
  // knots evenly spaced over [0, 1); output = the first unit = u (its cap is above any input): the
  // identity, i.e. plain linear range reduction (the root used when no training is asked for)
  for (int h = 0; h < kMlpHidden; h++) {
    w.w1[h] = 1.0f;
    w.b1[h] = -static_cast<float>(h) / kMlpHidden;
    w.w2[h] = h == 0 ? 1.0f : 0.0f;
    w.cap[h] = h == 0 ? 4.0f : 1.0f / kMlpHidden;
  }
  w.b2 = 0.0f;
}

}  // namespace

int mlp_grad_host(const float* d_u, const float* d_ulo, const float* d_t, size_t n,
                  const float* w_host, float* grad_host, double* loss_host, cudaStream_t st) {
  if (n >= (size_t(1) << 32)) return PLANB_EINVAL;
  DevBuf part, wb, gb, lb;
  if (!part.alloc(kGradBlocks * kRow * sizeof(float), nullptr) ||
      !wb.alloc(kMlpWeights * sizeof(float), nullptr) ||
      !gb.alloc(kMlpParams * sizeof(float), nullptr) || !lb.alloc(sizeof(double), nullptr)) {
    cudaGetLastError();
    return PLANB_ENOMEM;
  }
  if (cudaMemcpyAsync(wb.p, w_host, kMlpWeights * sizeof(float), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return PLANB_ECUDA;
  mlp_grad_kernel<<<kGradBlocks, kGradThreads, 0, st>>>(d_u, d_ulo, d_t,
                                                        static_cast<uint32_t>(n), wb.as<float>(),
                                                        part.as<float>());
  reduce_kernel<<<1, 64, 0, st>>>(part.as<float>(), kGradBlocks, static_cast<uint32_t>(n),
                                  gb.as<float>(), lb.as<double>());
  if (cudaGetLastError() != cudaSuccess) return PLANB_ECUDA;
  if (cudaMemcpyAsync(grad_host, gb.p, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(loss_host, lb.p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PLANB_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int knot_step_host(const float* d_u, const float* d_ulo, const float* d_t, size_t n,
                   float* w_host, const float* c_host, float* v_host, float* m_host,
                   float* q_host, int32_t step, float lr, double* loss_host, cudaStream_t st) {
  if (n >= (size_t(1) << 32) || step < 0) return PLANB_EINVAL;
  constexpr size_t kK = kMlpHidden + 1;
  DevBuf part, wb, vb, mb, qb, cb, sb, lb;
  if (!part.alloc(kGradBlocks * kRow * sizeof(float), nullptr) ||
      !wb.alloc(kMlpWeights * sizeof(float), nullptr) || !vb.alloc(kK * sizeof(float), nullptr) ||
      !mb.alloc(kK * sizeof(float), nullptr) || !qb.alloc(kK * sizeof(float), nullptr) ||
      !cb.alloc(kK * sizeof(float), nullptr) || !sb.alloc(sizeof(int), nullptr) ||
      !lb.alloc(sizeof(double), nullptr)) {
    cudaGetLastError();
    return PLANB_ENOMEM;
  }
  const int s0 = step;
  const bool ok =
      cudaMemcpyAsync(wb.p, w_host, kMlpWeights * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
      cudaMemcpyAsync(vb.p, v_host, kK * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
      cudaMemcpyAsync(mb.p, m_host, kK * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
      cudaMemcpyAsync(qb.p, q_host, kK * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
      cudaMemcpyAsync(cb.p, c_host, kK * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
      cudaMemcpyAsync(sb.p, &s0, sizeof(int), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) return PLANB_ECUDA;
  // one iteration of the training graph: the gradient, then the knot-value Adam update
  mlp_grad_kernel<<<kGradBlocks, kGradThreads, 0, st>>>(d_u, d_ulo, d_t, static_cast<uint32_t>(n),
                                                        wb.as<float>(), part.as<float>());
  knot_adam_kernel<<<1, 64, 0, st>>>(part.as<float>(), kGradBlocks, static_cast<uint32_t>(n),
                                     wb.as<float>(), vb.as<float>(), mb.as<float>(),
                                     qb.as<float>(), cb.as<float>(), sb.as<int>(), lr,
                                     lb.as<double>());
  if (cudaGetLastError() != cudaSuccess) return PLANB_ECUDA;
  if (cudaMemcpyAsync(w_host, wb.p, kMlpWeights * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(v_host, vb.p, kK * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(m_host, mb.p, kK * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(q_host, qb.p, kK * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(loss_host, lb.p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PLANB_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int mlp_forward_host(const float* d_u, size_t n, const float* w_host, float* d_y, cudaStream_t st) {
  if (n >= (size_t(1) << 32)) return PLANB_EINVAL;
  if (n == 0) return PLANB_OK;
  MlpWeights w;
  std::copy(w_host, w_host + kMlpHidden, w.w1);
  std::copy(w_host + kMlpHidden, w_host + 2 * kMlpHidden, w.b1);
  std::copy(w_host + 2 * kMlpHidden, w_host + 3 * kMlpHidden, w.w2);
  w.b2 = w_host[3 * kMlpHidden];
  std::copy(w_host + kMlpParams, w_host + kMlpWeights, w.cap);
  const uint32_t blocks = static_cast<uint32_t>(std::min<size_t>((n + 255) / 256, 4096));
  mlp_forward_kernel<<<blocks, 256, 0, st>>>(d_u, static_cast<uint32_t>(n), w, d_y);
  return cudaGetLastError() == cudaSuccess ? PLANB_OK : PLANB_ECUDA;
}

int build_learned(const Intervals& iv, uint32_t span, uint32_t leaves, uint32_t iters, float lr,
                  uint32_t max_window, LearnedBuild& out) {
  auto t0 = std::chrono::steady_clock::now();
  const uint64_t m = iv.size();
  const uint64_t n64 = m > 0 ? m - 1 : 0;       // finite keys: the inclusive ends start[i+1] - 1
  if (n64 >= (uint64_t(1) << 24)) return PLANB_EINVAL;   // ranks must stay exact in FP32
  const uint32_t n = static_cast<uint32_t>(n64);
  out = LearnedBuild();
  LearnedParams& P = out.P;
  init_weights(P.mlp);
  P.leaves = std::max<uint32_t>(1, leaves);
  P.span = span;
  P.inv_span = 1.0f / static_cast<float>(span);
  P.n_keys = static_cast<uint32_t>(m);           // counts range over [0, m - 1]
  out.leaves.assign(P.leaves, LeafModel{0, 0.0f, 0.0f});
  out.err.assign(P.leaves, kLeafFallback);
  if (n < 2) return PLANB_OK;                    // nothing to learn: every leaf takes the tree path
  std::vector<uint64_t> khi(n);
  for (uint32_t i = 0; i < n; i++) khi[i] = hi64(iv.start[i + 1] - 1);
  P.kmin = khi[0];
  const uint64_t range = khi[n - 1] - khi[0];
  P.inv_range = range ? 1.0f / static_cast<float>(range) : 0.0f;
  std::vector<float> hu(n), hl(n), ht(n);
  for (uint32_t i = 0; i < n; i++) {
    split_input(khi[i] - P.kmin, P.inv_range, &hu[i], &hl[i]);
    ht[i] = (static_cast<float>(i) + 0.5f) / static_cast<float>(n);
  }
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PLANB_ECUDA;
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } sg{st};
  // knot-value state for training: knots c_0..c_16 at the inputs' quantiles, values v_h = the CDF
  float c[kMlpHidden + 1], v0[kMlpHidden + 1];
  if (iters > 0) {
    for (int h = 0; h <= kMlpHidden; h++) {
      const size_t i = std::min<size_t>(n - 1, (static_cast<size_t>(h) * n) / kMlpHidden);
      c[h] = hu[i] + hl[i];
      v0[h] = (static_cast<float>(i) + 0.5f) / static_cast<float>(n);
    }
    c[kMlpHidden] = hu[n - 1] + hl[n - 1];
    v0[kMlpHidden] = 1.0f;
    for (int h = 1; h <= kMlpHidden; h++)     // strictly increasing knots (one float step apart)
      if (!(c[h] > c[h - 1])) c[h] = nextafterf(c[h - 1], 2.0f);
    for (int h = 0; h < kMlpHidden; h++) {
      P.mlp.w1[h] = 1.0f;
      P.mlp.b1[h] = -c[h];
      P.mlp.w2[h] = (v0[h + 1] - v0[h]) / (c[h + 1] - c[h]);
      // the last unit keeps rising past c_16 (addresses above the largest key)
      P.mlp.cap[h] = h + 1 < kMlpHidden ? c[h + 1] - c[h] : 4.0f;
    }
    P.mlp.b2 = v0[0];
  }
  DevBuf dk, du, dl, dt, dpart, dw, dm, dq, dv, dc, dstep, dloss, dleaf, dleaves, derr;
  if (!dk.alloc(n * 8ull, nullptr) || !du.alloc(n * 4ull, nullptr) ||
      !dl.alloc(n * 4ull, nullptr) || !dt.alloc(n * 4ull, nullptr) ||
      !dpart.alloc(kGradBlocks * kRow * 4ull, nullptr) || !dw.alloc(kMlpWeights * 4, nullptr) ||
      !dm.alloc(kRow * 4, nullptr) || !dq.alloc(kRow * 4, nullptr) ||
      !dv.alloc(kRow * 4, nullptr) || !dc.alloc(kRow * 4, nullptr) ||
      !dstep.alloc(sizeof(int), nullptr) || !dloss.alloc(sizeof(double), nullptr) ||
      !dleaf.alloc(n * 4ull, nullptr) || !dleaves.alloc(P.leaves * sizeof(LeafModel), nullptr) ||
      !derr.alloc(P.leaves * 4ull, nullptr)) {
    cudaGetLastError();
    return PLANB_ENOMEM;
  }
  float w0[kMlpWeights];
  std::copy(P.mlp.w1, P.mlp.w1 + kMlpHidden, w0);
  std::copy(P.mlp.b1, P.mlp.b1 + kMlpHidden, w0 + kMlpHidden);
  std::copy(P.mlp.w2, P.mlp.w2 + kMlpHidden, w0 + 2 * kMlpHidden);
  w0[3 * kMlpHidden] = P.mlp.b2;
  std::copy(P.mlp.cap, P.mlp.cap + kMlpHidden, w0 + kMlpParams);
  bool ok = cudaMemcpyAsync(dk.p, khi.data(), n * 8ull, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(du.p, hu.data(), n * 4ull, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(dl.p, hl.data(), n * 4ull, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(dt.p, ht.data(), n * 4ull, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(dw.p, w0, sizeof(w0), cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemsetAsync(dm.p, 0, kRow * 4, st) == cudaSuccess &&
            cudaMemsetAsync(dq.p, 0, kRow * 4, st) == cudaSuccess &&
            cudaMemsetAsync(dstep.p, 0, sizeof(int), st) == cudaSuccess;
  if (iters > 0)
    ok = ok &&
         cudaMemcpyAsync(dv.p, v0, sizeof(v0), cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(dc.p, c, sizeof(c), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) return PLANB_ECUDA;
  // loss before training
  mlp_grad_kernel<<<kGradBlocks, kGradThreads, 0, st>>>(du.as<float>(), dl.as<float>(),
                                                        dt.as<float>(), n, dw.as<float>(),
                                                        dpart.as<float>());
  reduce_kernel<<<1, 64, 0, st>>>(dpart.as<float>(), kGradBlocks, n, nullptr,
                                  dloss.as<double>());
  if (cudaMemcpyAsync(&out.loss0, dloss.p, sizeof(double), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return PLANB_ECUDA;
  // training: one graph holds `chunk` iterations (gradient, then update); replayed
  if (iters > 0) {
    const uint32_t chunk = std::min<uint32_t>(iters, 50);
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return PLANB_ECUDA;
    for (uint32_t it = 0; it < chunk; it++) {
      mlp_grad_kernel<<<kGradBlocks, kGradThreads, 0, st>>>(du.as<float>(), dl.as<float>(),
                                                        dt.as<float>(), n, dw.as<float>(),
                                                        dpart.as<float>());
      knot_adam_kernel<<<1, 64, 0, st>>>(dpart.as<float>(), kGradBlocks, n, dw.as<float>(),
                                         dv.as<float>(), dm.as<float>(), dq.as<float>(),
                                         dc.as<float>(), dstep.as<int>(), lr, dloss.as<double>());
      bump_step<<<1, 1, 0, st>>>(dstep.as<int>());
    }
    if (cudaStreamEndCapture(st, &graph) != cudaSuccess) return PLANB_ECUDA;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return PLANB_ECUDA;
    }
    bool gok = true;
    for (uint32_t done = 0; done < iters && gok; done += chunk)
      gok = cudaGraphLaunch(exec, st) == cudaSuccess;
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (!gok) return PLANB_ECUDA;
    out.iters = ((iters + chunk - 1) / chunk) * chunk;
  }
  // final loss with the trained weights
  mlp_grad_kernel<<<kGradBlocks, kGradThreads, 0, st>>>(du.as<float>(), dl.as<float>(),
                                                        dt.as<float>(), n, dw.as<float>(),
                                                        dpart.as<float>());
  reduce_kernel<<<1, 64, 0, st>>>(dpart.as<float>(), kGradBlocks, n, nullptr,
                                  dloss.as<double>());
  float w1[kMlpWeights];
  if (cudaMemcpyAsync(w1, dw.p, sizeof(w1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&out.loss, dloss.p, sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PLANB_ECUDA;
  std::copy(w1, w1 + kMlpHidden, P.mlp.w1);
  std::copy(w1 + kMlpHidden, w1 + 2 * kMlpHidden, P.mlp.b1);
  std::copy(w1 + 2 * kMlpHidden, w1 + 3 * kMlpHidden, P.mlp.w2);
  P.mlp.b2 = w1[3 * kMlpHidden];
  out.train_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                     .count();
  // leaves: route every key with the device arithmetic, fit each leaf on the host (least squares
  // of rank on the high half in double), then measure each leaf's error on the device
  const uint32_t gb = std::min<uint32_t>((n + 255) / 256, 4096);
  leaf_assign_kernel<<<gb, 256, 0, st>>>(dk.as<uint64_t>(), n, P, dleaf.as<uint32_t>());
  std::vector<uint32_t> leaf(n);
  if (cudaMemcpyAsync(leaf.data(), dleaf.p, n * 4ull, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PLANB_ECUDA;
  std::vector<uint64_t> base(P.leaves, ~0ull);
  std::vector<double> sx(P.leaves, 0), sy(P.leaves, 0), sxx(P.leaves, 0), sxy(P.leaves, 0);
  std::vector<uint32_t> cnt(P.leaves, 0);
  for (uint32_t i = 0; i < n; i++) base[leaf[i]] = std::min(base[leaf[i]], khi[i]);
  for (uint32_t i = 0; i < n; i++) {
    const uint32_t l = leaf[i];
    const double x = static_cast<double>(khi[i] - base[l]);
    const double y = static_cast<double>(i);
    sx[l] += x; sy[l] += y; sxx[l] += x * x; sxy[l] += x * y; cnt[l]++;
  }
  std::vector<double> la(P.leaves, 0.0), ls(P.leaves, 0.0);
  for (uint32_t l = 0; l < P.leaves; l++) {
    if (!cnt[l]) continue;
    const double c = cnt[l];
    const double var = sxx[l] - sx[l] * sx[l] / c;
    const double slope = var > 0 ? std::max((sxy[l] - sx[l] * sy[l] / c) / var, 0.0) : 0.0;
    ls[l] = slope;
    la[l] = (sy[l] - slope * sx[l]) / c;
  }
  // The bound a leaf records is its largest |predicted - true rank|: shift each least-squares line
  // to the middle of its residuals' range, which halves the spread the bound must cover when the
  // residuals are lopsided (a step in the key distribution).
  std::vector<double> rmin(P.leaves, 0.0), rmax(P.leaves, 0.0);
  std::vector<uint8_t> seen(P.leaves, 0);
  for (uint32_t i = 0; i < n; i++) {
    const uint32_t l = leaf[i];
    const double r = static_cast<double>(i) -
                     (la[l] + ls[l] * static_cast<double>(khi[i] - base[l]));
    if (!seen[l]) {
      rmin[l] = rmax[l] = r;
      seen[l] = 1;
    } else {
      rmin[l] = std::min(rmin[l], r);
      rmax[l] = std::max(rmax[l], r);
    }
  }
  for (uint32_t l = 0; l < P.leaves; l++) {
    LeafModel& lm = out.leaves[l];
    if (!cnt[l]) continue;
    lm.base = base[l];
    lm.s = static_cast<float>(ls[l]);
    lm.a = static_cast<float>(la[l] + 0.5 * (rmin[l] + rmax[l]));
  }
  if (cudaMemcpyAsync(dleaves.p, out.leaves.data(), P.leaves * sizeof(LeafModel),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(derr.p, 0, P.leaves * 4ull, st) != cudaSuccess)
    return PLANB_ECUDA;
  leaf_error_kernel<<<gb, 256, 0, st>>>(dk.as<uint64_t>(), n, P, dleaves.as<LeafModel>(),
                                        derr.as<uint32_t>());
  std::vector<uint32_t> e(P.leaves);
  if (cudaMemcpyAsync(e.data(), derr.p, P.leaves * 4ull, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PLANB_ECUDA;
  uint64_t covered = 0;
  double esum = 0;
  for (uint32_t l = 0; l < P.leaves; l++) {
    if (!cnt[l]) continue;
    const uint32_t bound = e[l] + 1;             // + 1: addresses between two keys
    out.max_err = std::max(out.max_err, bound);
    if (bound <= max_window) {
      out.err[l] = static_cast<uint16_t>(bound);
      covered += cnt[l];
      esum += static_cast<double>(bound) * cnt[l];
    }
  }
  out.covered = static_cast<double>(covered) / n;
  out.mean_err = covered ? esum / covered : 0.0;
  out.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                     .count();
  return PLANB_OK;
}

}  // namespace planb
