// Learned (q, p) predictor: a 3-layer MLP (F = 12 -> 64 -> 64 -> 15, ReLU)
// whose 15 outputs estimate log10 of the excess rank-k error that each
// (q, p), q in {0..4}, p in {5, 10, 20}, would reach (pair j = 3 qi + pi),
// trained by mean squared error with Adam; the features of a probe sketch;
// and the selection that turns the estimates into (q, p): the cheapest pair,
// by cost (2q + 2)(k + p), whose estimate plus a calibrated margin delta
// stays within the request.
//
// Parameter layout (flat FP32): W1 (F x H, row-major), b1 (H), W2 (H x H),
// b2 (H), W3 (H x 15), b3 (15), delta (1, log10 units; its gradient is 0).
//
// Training step = mlp_sample_kernel<true> (one CTA of H threads per sample:
// forward and per-sample backward quantities) + mlp_grad_reduce_kernel (one
// thread per parameter summing the per-sample terms in sample order, so
// gradients are deterministic) + adam_kernel.
#include <cmath>

#include "common.cuh"

namespace rqlp {
namespace {

constexpr int F = RQLP_MLP_FEATURES;
constexpr int H = RQLP_MLP_HIDDEN;
constexpr int NQ = 5, NP = 3, NO = RQLP_MLP_OUTPUTS;
static_assert(NO == NQ * NP, "one output per (q, p)");
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + F * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * NO, OFF_DELTA = OFF_B3 + NO, NPARAM = OFF_DELTA + 1;
static_assert(NPARAM == RQLP_MLP_PARAMS, "parameter count");

__device__ const int kQChoices[NQ] = {0, 1, 2, 3, 4};
__device__ const int kPChoices[NP] = {5, 10, 20};

// Per-sample buffers of a training step (B samples).
struct SampleBufs {
  float *h1, *h2, *dz1, *dz2, *d3, *loss;
};

template <bool BACKWARD>
__global__ void __launch_bounds__(H)
mlp_sample_kernel(const float* __restrict__ prm, const float* __restrict__ X, int B, const float* __restrict__ Y,
                  float* __restrict__ est, SampleBufs sb) {
  __shared__ float x[F], h1[H], h2[H], d3[NO], dz2[H], sq[NO];
  const int t = threadIdx.x;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    if (t < F) x[t] = X[(int64_t)b * F + t];
    __syncthreads();
    float z1 = prm[OFF_B1 + t];
#pragma unroll
    for (int f = 0; f < F; ++f) z1 += x[f] * prm[OFF_W1 + f * H + t];
    h1[t] = z1 > 0.f ? z1 : 0.f;
    __syncthreads();
    float z2 = prm[OFF_B2 + t];
    for (int j = 0; j < H; ++j) z2 += h1[j] * prm[OFF_W2 + j * H + t];
    h2[t] = z2 > 0.f ? z2 : 0.f;
    __syncthreads();
    if (t < NO) {
      float o = prm[OFF_B3 + t];
      for (int j = 0; j < H; ++j) o += h2[j] * prm[OFF_W3 + j * NO + t];
      if (!BACKWARD) est[(int64_t)b * NO + t] = o;
      if (BACKWARD) {
        // d(mean of squares)/d(estimate) for this sample's output t
        const float r = o - Y[(int64_t)b * NO + t];
        d3[t] = 2.f * r / (float)(B * NO);
        sq[t] = r * r;
      }
    }
    __syncthreads();
    if (BACKWARD) {
      if (t == 0) {
        float s = 0.f;
        for (int o = 0; o < NO; ++o) s += sq[o];
        sb.loss[b] = s / (float)NO;
      }
      if (t < NO) sb.d3[(int64_t)b * NO + t] = d3[t];
      float dh2 = 0.f;
#pragma unroll
      for (int o = 0; o < NO; ++o) dh2 += d3[o] * prm[OFF_W3 + t * NO + o];
      const float g2 = z2 > 0.f ? dh2 : 0.f;
      dz2[t] = g2;
      sb.h1[(int64_t)b * H + t] = h1[t];
      sb.h2[(int64_t)b * H + t] = h2[t];
      sb.dz2[(int64_t)b * H + t] = g2;
      __syncthreads();
      float dh1 = 0.f;
      for (int j = 0; j < H; ++j) dh1 += dz2[j] * prm[OFF_W2 + t * H + j];
      sb.dz1[(int64_t)b * H + t] = z1 > 0.f ? dh1 : 0.f;
    }
    __syncthreads();
  }
}

// grad[i] = sum over samples b (in order) of the per-sample term of parameter i.
__global__ void mlp_grad_reduce_kernel(const float* __restrict__ X, int B, SampleBufs sb, float* __restrict__ grad,
                                       float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == NPARAM && loss != nullptr) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += sb.loss[b];
    *loss = s / (float)B;
  }
  if (i >= NPARAM) return;
  float s = 0.f;
  if (i < OFF_B1) {
    const int f = (i - OFF_W1) / H, h = (i - OFF_W1) % H;
    for (int b = 0; b < B; ++b) s += X[(int64_t)b * F + f] * sb.dz1[(int64_t)b * H + h];
  } else if (i < OFF_W2) {
    const int h = i - OFF_B1;
    for (int b = 0; b < B; ++b) s += sb.dz1[(int64_t)b * H + h];
  } else if (i < OFF_B2) {
    const int j = (i - OFF_W2) / H, h = (i - OFF_W2) % H;
    for (int b = 0; b < B; ++b) s += sb.h1[(int64_t)b * H + j] * sb.dz2[(int64_t)b * H + h];
  } else if (i < OFF_W3) {
    const int h = i - OFF_B2;
    for (int b = 0; b < B; ++b) s += sb.dz2[(int64_t)b * H + h];
  } else if (i < OFF_B3) {
    const int h = (i - OFF_W3) / NO, o = (i - OFF_W3) % NO;
    for (int b = 0; b < B; ++b) s += sb.h2[(int64_t)b * H + h] * sb.d3[(int64_t)b * NO + o];
  } else if (i < OFF_DELTA) {
    const int o = i - OFF_B3;
    for (int b = 0; b < B; ++b) s += sb.d3[(int64_t)b * NO + o];
  }   // delta: 0 (set by calibration)
  grad[i] = s;
}

__global__ void adam_kernel(float* __restrict__ prm, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int n, float lr, float beta1, float beta2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = beta1 * m1[i] + (1.f - beta1) * gi;
  const float v = beta2 * m2[i] + (1.f - beta2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  prm[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// Features of the probe R-diagonal (R w x w upper, ldr): see probe_features
// in the FP64 reference. One warp.
__global__ void probe_features_kernel(const float* __restrict__ R, int64_t ldr, int w, int k, int64_t mn,
                                      float* __restrict__ feat) {
  __shared__ float lr[RQLP_MAX_D];
  const int t = threadIdx.x;
  const float r0 = R[0];
  for (int i = t; i < w; i += 32) lr[i] = log10f(fmaxf(R[(int64_t)i * ldr + i], 1e-30f) / r0);
  __syncwarp();
  // std of the steps lr[i+1] - lr[i]
  float s = 0.f, s2 = 0.f;
  for (int i = t; i + 1 < w; i += 32) {
    const float st = lr[i + 1] - lr[i];
    s += st;
    s2 += st * st;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if (t == 0) {
    auto L = [&](int i) { return lr[min(max(i, 1), w) - 1]; };
    const int h = (k + 1) / 2;
    const int ns = w - 1;
    float sd = 0.f;
    if (ns > 0) {
      const float mu = s / ns;
      sd = sqrtf(fmaxf(s2 / ns - mu * mu, 0.f));
    }
    feat[0] = L(k);
    feat[1] = L(h);
    feat[2] = L(k) - L(h);
    feat[3] = L(k + 1) - L(k);
    feat[4] = L(k + 5) - L(k);
    feat[5] = L(k + 10) - L(k);
    feat[6] = L(k + 20) - L(k);
    feat[7] = L(k + 20) - L(k + 10);
    feat[8] = sd;
    feat[9] = log10f((float)k);
    feat[10] = log10f((float)mn);
    feat[11] = (float)k / (float)mn;
  }
}

// (q, p) for one sample: the cheapest pair (cost (2q + 2)(k + p); ties
// smaller q, then smaller p) with est + delta <= log10(target); (4, 20) when
// none qualifies; (2, 10) when the probe failed (status != 0) or an estimate
// or delta is not finite.
__global__ void predict_kernel(const float* __restrict__ est, const float* __restrict__ prm, const int* __restrict__ info,
                               float log_target, int k, int* __restrict__ qp) {
  const float delta = prm[OFF_DELTA];
  bool ok = (info == nullptr || info[0] == 0) && isfinite(delta);
  for (int o = 0; o < NO; ++o) ok = ok && isfinite(est[o]);
  if (!ok) {
    qp[0] = 2;
    qp[1] = 10;
    return;
  }
  int bq = NQ - 1, bp = NP - 1;
  long long best = -1;
  for (int qi = 0; qi < NQ; ++qi)
    for (int pi = 0; pi < NP; ++pi) {
      if (est[qi * NP + pi] + delta > log_target) continue;
      const long long c = (long long)(2 * kQChoices[qi] + 2) * (k + kPChoices[pi]);
      if (best < 0 || c < best) {   // the loops run q, then p, upwards: the first minimum wins ties
        best = c;
        bq = qi;
        bp = pi;
      }
    }
  qp[0] = kQChoices[bq];
  qp[1] = kPChoices[bp];
}

SampleBufs carve(void* ws, int B) {
  SampleBufs sb;
  float* p = static_cast<float*>(ws);
  sb.h1 = p;
  sb.h2 = sb.h1 + (size_t)B * H;
  sb.dz1 = sb.h2 + (size_t)B * H;
  sb.dz2 = sb.dz1 + (size_t)B * H;
  sb.d3 = sb.dz2 + (size_t)B * H;
  sb.loss = sb.d3 + (size_t)B * NO;
  return sb;
}

}  // namespace

size_t mlp_workspace_floats(int B) { return (size_t)B * (4 * H + NO + 1); }

cudaError_t mlp_forward(const float* prm, const float* X, int B, float* est, cudaStream_t st) {
  const int blocks = std::min(B, sm_count() * 8);
  mlp_sample_kernel<false><<<blocks, H, 0, st>>>(prm, X, B, nullptr, est, SampleBufs{});
  note_launch();
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float* prm, const float* X, const float* Y, int B, float* grad, float* loss, void* ws,
                     cudaStream_t st) {
  SampleBufs sb = carve(ws, B);
  const int blocks = std::min(B, sm_count() * 8);
  mlp_sample_kernel<true><<<blocks, H, 0, st>>>(prm, X, B, Y, nullptr, sb);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mlp_grad_reduce_kernel<<<(NPARAM + 1 + 127) / 128, 128, 0, st>>>(X, B, sb, grad, loss);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* prm, const float* g, float* m1, float* m2, int n, float lr, float beta1, float beta2,
                     float eps, int step, cudaStream_t st) {
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(prm, g, m1, m2, n, lr, beta1, beta2, eps, c1, c2);
  note_launch();
  return cudaGetLastError();
}

cudaError_t probe_features(const float* R, int64_t ldr, int w, int k, int64_t mn, float* feat, cudaStream_t st) {
  probe_features_kernel<<<1, 32, 0, st>>>(R, ldr, w, k, mn, feat);
  note_launch();
  return cudaGetLastError();
}

cudaError_t predict_qp(const float* est, const float* prm, const int* info, double target, int k, int* qp,
                       cudaStream_t st) {
  predict_kernel<<<1, 1, 0, st>>>(est, prm, info, (float)std::log10(target), k, qp);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rqlp
