// Evaluation utilities on the device (section 5.2 and section 4.1):
//
//  * rank-r errors ||A - A_r||_F for r = 1..d with A_r = Q L(:, 1:r) P(:, 1:r)^T,
//    from the projection identity ||A - A_r||_F^2 = ||A||_F^2 - ||L(:, 1:r)||_F^2
//    (A_r = A P_r P_r^T for this chain), and the explicit residual for one r
//    (a pass over A that subtracts the rank-r product tile by tile);
//  * the canonical angles between two subspaces given by orthonormal bases X
//    (rows x a) and Y (rows x b): the sines, singular values of (I - X X^T) Y,
//    or the cosines, singular values of X^T Y (Theorem 2's distances), from
//    the eigenvalues of their b x b Gram matrix (FP64) by cyclic Jacobi.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rqlp {
namespace {

// errs[r - 1] = sqrt(max(||A||^2 - sum_{j < r} ||L(:, j)||^2, 0)); one CTA.
__global__ void rank_errors_kernel(const float* __restrict__ L, int64_t ldl, int d, const double* __restrict__ normA2,
                                   double* __restrict__ errs) {
  __shared__ double col[RQLP_MAX_D];
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int i = j; i < d; ++i) {   // L is lower triangular
      const double v = L[(int64_t)i * ldl + j];
      s += v * v;
    }
    col[j] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    const double a2 = *normA2;
    for (int r = 0; r < d; ++r) {
      acc += col[r];
      errs[r] = sqrt(fmax(a2 - acc, 0.0));
    }
  }
}

// sum over a 64 x 64 tile of A of (A - W P^T)^2, W (m x r), P (n x r); r <= 256.
constexpr int RT = 64, RK = 32;
__global__ void __launch_bounds__(256)
rank_residual_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float* __restrict__ W,
                     int64_t ldw, const float* __restrict__ P, int64_t ldp, int r, double* __restrict__ out) {
  __shared__ float Ws[RK][RT + 1], Ps[RK][RT + 1];
  const int64_t i0 = (int64_t)blockIdx.y * RT, j0 = (int64_t)blockIdx.x * RT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 4 x 4 outputs per thread
  float acc[4][4] = {};
  for (int k0 = 0; k0 < r; k0 += RK) {
    for (int e = threadIdx.x; e < RT * RK; e += 256) {
      const int row = e / RK, kk = e % RK;
      const int64_t gi = i0 + row, gj = j0 + row;
      Ws[kk][row] = (gi < m && k0 + kk < r) ? W[gi * ldw + k0 + kk] : 0.f;
      Ps[kk][row] = (gj < n && k0 + kk < r) ? P[gj * ldp + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < RK; ++kk) {
      float w[4], p[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        w[t] = Ws[kk][ty * 4 + t];
        p[t] = Ps[kk][tx * 4 + t];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(w[a], p[b], acc[a][b]);
    }
    __syncthreads();
  }
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
      if (gi < m && gj < n) {
        const double e = (double)A[gi * lda + gj] - (double)acc[a][b];
        s += e * e;
      }
    }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(out, t);
  }
}

__global__ void sqrt_kernel(double* x) { *x = sqrt(fmax(*x, 0.0)); }

// G (b x b, FP64, symmetric) = R^T R for R (rows x b, FP32, ldr).
__global__ void gram64_kernel(const float* __restrict__ R, int64_t rows, int b, int64_t ldr, double* __restrict__ G) {
  const int i = blockIdx.y, j0 = blockIdx.x * blockDim.x;
  const int j = j0 + threadIdx.x;
  if (j < i || j >= b) return;   // upper triangle, mirrored below
  double s = 0.0;
  for (int64_t t = 0; t < rows; ++t) s += (double)R[t * ldr + i] * (double)R[t * ldr + j];
  G[(int64_t)i * b + j] = s;
  G[(int64_t)j * b + i] = s;
}

// Eigenvalues of the symmetric b x b matrix S (FP64, global, overwritten) by
// cyclic Jacobi with the round-robin pair order (b / 2 disjoint rotations per
// round, applied to the rows, then to the columns); out = sqrt of the
// eigenvalues (clipped at 0), largest first. One CTA.
__global__ void __launch_bounds__(256) jacobi_sqrt_eig_kernel(double* __restrict__ S, int b, double* __restrict__ out) {
  extern __shared__ double sh[];
  const int nb = b + (b & 1);                 // even order: a dummy index b when b is odd
  double* cs = sh;                            // [nb / 2] cosines
  double* sn = cs + nb / 2;                   // [nb / 2] sines
  int* top = reinterpret_cast<int*>(sn + nb / 2);
  int* bot = top + nb / 2;
  __shared__ int done;
  const int npairs = nb / 2;
  for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
    top[t] = 2 * t;
    bot[t] = 2 * t + 1;
  }
  __syncthreads();
  auto at = [&](int i, int j) -> double& { return S[(int64_t)i * b + j]; };
  for (int sweep = 0; sweep < 30; ++sweep) {
    double part = 0.0, diag = 0.0;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const double v = S[e];
      if (e / b != e % b) part += v * v;
      else diag += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      part += __shfl_down_sync(0xffffffffu, part, o);
      diag += __shfl_down_sync(0xffffffffu, diag, o);
    }
    __shared__ double po[8], pd[8];
    if ((threadIdx.x & 31) == 0) {
      po[threadIdx.x >> 5] = part;
      pd[threadIdx.x >> 5] = diag;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double so = 0.0, sd = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        so += po[w];
        sd += pd[w];
      }
      // off-diagonal Frobenius norm at 1e-13 of the whole: every eigenvalue
      // then sits within 1e-13 ||S||_F of the diagonal (Weyl)
      done = (so <= 1e-26 * (sd + so)) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int round = 0; round < nb - 1; ++round) {
      for (int t = threadIdx.x; t < npairs; t += blockDim.x) {   // rotation of pair t
        int p = top[t], q = bot[t];
        if (p > q) { const int x = p; p = q; q = x; }
        double c = 1.0, s = 0.0;
        if (q < b && p != q) {
          const double apq = at(p, q);
          if (apq != 0.0) {
            const double tau = (at(q, q) - at(p, p)) / (2.0 * apq);
            const double tt = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        cs[t] = c;
        sn[t] = s;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < npairs * b; e += blockDim.x) {   // rows p, q
        const int t = e / b, j = e % b;
        int p = top[t], q = bot[t];
        if (p > q) { const int x = p; p = q; q = x; }
        if (q >= b || sn[t] == 0.0) continue;
        const double a = at(p, j), bq = at(q, j);
        at(p, j) = cs[t] * a - sn[t] * bq;
        at(q, j) = sn[t] * a + cs[t] * bq;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < npairs * b; e += blockDim.x) {   // columns p, q
        const int t = e / b, i = e % b;
        int p = top[t], q = bot[t];
        if (p > q) { const int x = p; p = q; q = x; }
        if (q >= b || sn[t] == 0.0) continue;
        const double a = at(i, p), bq = at(i, q);
        at(i, p) = cs[t] * a - sn[t] * bq;
        at(i, q) = sn[t] * a + cs[t] * bq;
      }
      __syncthreads();
      if (threadIdx.x == 0 && npairs > 1) {   // round-robin: index 0 stays, the others move one place
        const int last_top = top[npairs - 1], first_bot = bot[0];
        for (int t = npairs - 1; t > 1; --t) top[t] = top[t - 1];
        top[1] = first_bot;
        for (int t = 0; t < npairs - 1; ++t) bot[t] = bot[t + 1];
        bot[npairs - 1] = last_top;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {   // sorted largest first (b <= 256: insertion sort)
    for (int i = 0; i < b; ++i) out[i] = sqrt(fmax(at(i, i), 0.0));
    for (int i = 1; i < b; ++i) {
      const double v = out[i];
      int j = i - 1;
      while (j >= 0 && out[j] < v) {
        out[j + 1] = out[j];
        --j;
      }
      out[j + 1] = v;
    }
  }
}

// R = Y - T (rows x b).
// R = Y - T; R may be T (each entry is read and written by the same thread).
__global__ void sub_kernel(int64_t rows, int b, const float* __restrict__ Y, int64_t ldy, const float* T,
                           int64_t ldt, float* R, int64_t ldr) {
  const int64_t total = rows * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b, j = e % b;
    R[i * ldr + j] = Y[i * ldy + j] - T[i * ldt + j];
  }
}

}  // namespace
}  // namespace rqlp

using namespace rqlp;

extern "C" {

rqlp_status rqlp_rank_errors(const float* L, int64_t ldl, int d, const double* d_diag, double* errs, void* stream) {
  if (L == nullptr || d_diag == nullptr || errs == nullptr || d < 1 || d > RQLP_MAX_D || ldl < d) return RQLP_ERR_ARG;
  rank_errors_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(L, ldl, d, d_diag, errs);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_rank_residual_workspace_bytes(int64_t m, int r) {
  if (m <= 0 || r < 1 || r > RQLP_MAX_D) return 0;
  return (size_t)round_up((int64_t)(m * round_up(r, 4) * sizeof(float)), 256);
}

rqlp_status rqlp_rank_residual(const float* A, int64_t m, int64_t n, int64_t lda, const float* Q, int64_t ldq,
                               const float* L, int64_t ldl, int d, const float* P, int64_t ldp, int r, double* out,
                               void* workspace, size_t ws_bytes, void* stream) {
  if (A == nullptr || Q == nullptr || L == nullptr || P == nullptr || out == nullptr || m <= 0 || n <= 0 ||
      d < 1 || d > RQLP_MAX_D || r < 1 || r > d || lda < n || ldq < d || ldl < d || ldp < d)
    return RQLP_ERR_ARG;
  if (workspace == nullptr || ws_bytes < rqlp_rank_residual_workspace_bytes(m, r) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return RQLP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* W = static_cast<float*>(workspace);
  const int64_t ldw = round_up(r, 4);
  // W = Q L(:, 1:r)  (m x r)
  if (gemm_f32_ex(false, m, r, d, Q, ldq, L, ldl, W, ldw, 1, nullptr, nullptr, nullptr, kGateNone, false, st) !=
      cudaSuccess)
    return RQLP_ERR_CUDA;
  if (cudaMemsetAsync(out, 0, sizeof(double), st) != cudaSuccess) return RQLP_ERR_CUDA;
  dim3 grid((unsigned)cdiv(n, RT), (unsigned)cdiv(m, RT));
  rank_residual_kernel<<<grid, 256, 0, st>>>(A, m, n, lda, W, ldw, P, ldp, r, out);
  sqrt_kernel<<<1, 1, 0, st>>>(out);
  note_launch(2);
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_subspace_workspace_bytes(int64_t rows, int a, int b) {
  if (rows <= 0 || a < 1 || b < 1 || a > RQLP_MAX_D || b > RQLP_MAX_D || b > rows) return 0;
  Arena ar;
  ar.dry = true;
  ar.take<float>((size_t)a * round_up(b, 4));       // M = X^T Y
  ar.take<float>((size_t)rows * round_up(b, 4));    // T = X M, then R = Y - T
  ar.take<float>(gemm_f32_part_floats(a, b, rows));
  ar.take<double>((size_t)b * b);                  // Gram
  return ar.off;
}

rqlp_status rqlp_subspace_angles(const float* X, int64_t rows, int a, int64_t ldx, const float* Y, int b,
                                 int64_t ldy, int cosines, double* out, void* workspace, size_t ws_bytes,
                                 void* stream) {
  const size_t need = rqlp_subspace_workspace_bytes(rows, a, b);
  if (need == 0 || X == nullptr || Y == nullptr || out == nullptr || ldx < a || ldy < b ||
      (cosines != 0 && cosines != 1))
    return RQLP_ERR_ARG;
  if (workspace == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return RQLP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena ar;
  ar.base = static_cast<char*>(workspace);
  ar.cap = ws_bytes;
  const int64_t ldb = round_up(b, 4);
  float* M = ar.take<float>((size_t)a * ldb);
  float* T = ar.take<float>((size_t)rows * ldb);
  float* part = ar.take<float>(gemm_f32_part_floats(a, b, rows));
  double* G = ar.take<double>((size_t)b * b);
  // M = X^T Y
  if (gemm_f32_ex(true, a, b, rows, X, ldx, Y, ldy, M, ldb, gemm_f32_splits(a, b, rows), part, nullptr, nullptr,
                  kGateNone, false, st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  if (cosines) {
    gram64_kernel<<<dim3((unsigned)cdiv(b, 128), (unsigned)b), 128, 0, st>>>(M, a, b, ldb, G);
  } else {
    // R = Y - X M, then G = R^T R
    if (gemm_f32_ex(false, rows, b, a, X, ldx, M, ldb, T, ldb, 1, nullptr, nullptr, nullptr, kGateNone, false, st) !=
        cudaSuccess)
      return RQLP_ERR_CUDA;
    const int blocks = (int)std::min<int64_t>(cdiv(rows * b, 256), (int64_t)sm_count() * 8);
    sub_kernel<<<blocks, 256, 0, st>>>(rows, b, Y, ldy, T, ldb, T, ldb);
    gram64_kernel<<<dim3((unsigned)cdiv(b, 128), (unsigned)b), 128, 0, st>>>(T, rows, b, ldb, G);
    note_launch();
  }
  const int nb = b + (b & 1);
  const size_t shm = (size_t)nb * sizeof(double) + (size_t)nb * sizeof(int);
  jacobi_sqrt_eig_kernel<<<1, 256, shm, st>>>(G, b, out);
  note_launch(2);
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

}  // extern "C"
