// d x d kernels of the chain: Cholesky factor and inverse for CholeskyQR,
// transposes, the L write-out and the diagnostics.
//
// chol_inv_kernel factors G = L D L^T by right-looking elimination on the
// augmented matrix [G | I] in one CTA: step j subtracts l_ij = G'_ji / G'_jj
// times row j from every row i > j, on both halves. The left half leaves the
// Schur complements (upper part, packed), the right half becomes L^{-1}
// (lower part, packed). Then R = D^{1/2} L^T and R^{-1} = L^{-T} D^{-1/2}.
// Rows i > j only read row j during step j, so one barrier per column
// suffices. A pivot that is not clearly positive restarts the elimination
// on G + s I (shifted CholeskyQR, Fukaya et al. 2020); the caller then runs
// one more CholeskyQR pass, gated on the flag this kernel raises.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rqlp {

namespace {

__host__ __device__ __forceinline__ int tri(int d) { return d * (d + 1) / 2; }
// Packed upper triangle, row-major: row i holds columns i..d-1.
__device__ __forceinline__ int iu(int d, int i, int l) { return i * d - i * (i - 1) / 2 + (l - i); }
// Packed lower triangle, row-major: row i holds columns 0..i.
__device__ __forceinline__ int il(int i, int t) { return i * (i + 1) / 2 + t; }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float u = 5.9604645e-8f; };
template <> struct Eps<double> { static constexpr double u = 1.1102230246251565e-16; };

__device__ void post_error(int* info, int code, int detail) {
  if (info != nullptr && atomicCAS(info, 0, code) == 0) info[1] = detail;
}

__device__ void write_identity(int d, float* R, float* Rinv, int64_t ldr) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, l = e % d;
    float v = i == l ? 1.f : 0.f;
    R[i * ldr + l] = v;
    Rinv[i * ldr + l] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024)
chol_inv_kernel(int d, const float* __restrict__ G, int64_t ldg, float* __restrict__ R,
                float* __restrict__ Rinv, int64_t ldr, int* info, double* shift_count,
                int* gate_out, const int* gate_in, T* gstore) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = gstore != nullptr ? gstore : reinterpret_cast<T*>(smem_raw);
  T* W = S + tri(d);
  __shared__ T s_red[32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  if (gate_in != nullptr && *gate_in == 0) {   // pass not needed: R = R^{-1} = I
    write_identity(d, R, Rinv, ldr);
    return;
  }

  // Trace of G sets the scale of the shift and exposes non-finite input.
  T tr = 0;
  for (int i = tid; i < d; i += blockDim.x) tr += (T)G[(int64_t)i * ldg + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
  if (lane == 0) s_red[warp] = tr;
  __syncthreads();
  T trace = 0;
  for (int w = 0; w < nwarps; ++w) trace += s_red[w];
  if (!isfinite(trace)) {
    if (tid == 0) post_error(info, RQLP_ERR_NONFINITE, 0);
    write_identity(d, R, Rinv, ldr);
    return;
  }
  const T shift = (T)(100.0 * d) * Eps<T>::u * trace;
  const T rel_tol = (T)64 * Eps<T>::u;

  int fail_col = -1;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const T sh = attempt == 0 ? (T)0 : shift;
    for (int i = warp; i < d; i += nwarps) {
      for (int l = i + lane; l < d; l += 32) {
        T v = (T)G[(int64_t)i * ldg + l];
        if (l == i) v += sh;
        S[iu(d, i, l)] = v;
      }
      for (int t = lane; t <= i; t += 32) W[il(i, t)] = (t == i) ? (T)1 : (T)0;
    }
    __syncthreads();
    fail_col = -1;
    for (int j = 0; j < d; ++j) {
      const T piv = S[iu(d, j, j)];
      const T g0 = (T)G[(int64_t)j * ldg + j] + sh;
      if (!(piv > rel_tol * g0) || !isfinite(piv)) { fail_col = j; break; }   // uniform
      const T pinv = (T)1 / piv;
      for (int i = j + 1 + warp; i < d; i += nwarps) {
        const T f = S[iu(d, j, i)] * pinv;
        for (int l = i + lane; l < d; l += 32) S[iu(d, i, l)] -= f * S[iu(d, j, l)];
        for (int t = lane; t <= j; t += 32) W[il(i, t)] -= f * W[il(j, t)];
      }
      __syncthreads();
    }
    if (fail_col < 0) break;
    __syncthreads();
    if (attempt == 0 && tid == 0) {
      if (gate_out != nullptr) *gate_out = 1;
      if (shift_count != nullptr) atomicAdd(shift_count, 1.0);
    }
  }

  if (fail_col >= 0) {   // breakdown even with the shift: report, stay finite
    if (tid == 0) post_error(info, RQLP_ERR_BREAKDOWN, fail_col + 1);
    write_identity(d, R, Rinv, ldr);
    return;
  }

  // R[i, l] = S[i, l] / sqrt(piv_i) (l >= i);  R^{-1}[i, l] = W[l, i] / sqrt(piv_l).
  for (int e = tid; e < d * d; e += blockDim.x) {
    int i = e / d, l = e % d;
    float rv = 0.f, iv = 0.f;
    if (l >= i) {
      rv = (float)(S[iu(d, i, l)] / sqrt(S[iu(d, i, i)]));
      iv = (float)(W[il(l, i)] / sqrt(S[iu(d, l, l)]));
    }
    R[(int64_t)i * ldr + l] = rv;
    Rinv[(int64_t)i * ldr + l] = iv;
  }
}

// Y = X^T for a d x d matrix.
__global__ void transpose_kernel(int d, const float* __restrict__ X, int64_t ldx, float* __restrict__ Y,
                                 int64_t ldy) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int i = e / d, l = e % d;
    Y[(int64_t)l * ldy + i] = X[(int64_t)i * ldx + l];
  }
}

// L = Rhat^T written as a full d x d block (strict upper part zero) and
// ||L||_F^2 accumulated into diag[1] (double, one atomic per CTA).
__global__ void write_L_kernel(int d, const float* __restrict__ Rh, int64_t ldrh, float* __restrict__ L,
                               int64_t ldl, double* diag) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int i = e / d, j = e % d;
    float v = j <= i ? Rh[(int64_t)j * ldrh + i] : 0.f;
    L[(int64_t)i * ldl + j] = v;
    acc += (double)v * (double)v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && diag != nullptr) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(&diag[1], s);
  }
}

// info <- 0, scratch scalars <- 0.
__global__ void init_kernel(int* info, int* gates, int ngates, double* scal, int nscal) {
  int t = threadIdx.x;
  if (t < 2) info[t] = 0;
  if (t < ngates) gates[t] = 0;
  if (t < nscal) scal[t] = 0.0;
}

// diag = [||A||^2, ||L||^2, ||A||^2 - ||L||^2, shifts]; flags non-finite A.
__global__ void finish_diag_kernel(const double* scal, double* diag, int* info) {
  if (threadIdx.x != 0) return;
  double a2 = scal[0], l2 = scal[1];
  if (!isfinite(a2)) post_error(info, RQLP_ERR_NONFINITE, 0);
  if (diag != nullptr) {
    diag[0] = a2;
    diag[1] = l2;
    diag[2] = a2 - l2;
    diag[3] = scal[2];
  }
}

__global__ void copy_kernel(int64_t rows, int64_t cols, const float* __restrict__ X, int64_t ldx,
                            float* __restrict__ Y, int64_t ldy) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / cols, c = e % cols;
    Y[r * ldy + c] = X[r * ldx + c];
  }
}

template <typename T>
size_t chol_smem_bytes(int d) { return (size_t)2 * tri(d) * sizeof(T); }

size_t smem_optin() {
  static size_t cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
      cached = (size_t)v;
    else
      cached = 48 * 1024;
  }
  return cached;
}

template <typename T>
cudaError_t launch_chol(int d, const float* G, int64_t ldg, float* R, float* Rinv, int64_t ldr, int* info,
                        double* shift_count, int* gate_out, const int* gate_in, void* gstore,
                        cudaStream_t st) {
  const size_t need = chol_smem_bytes<T>(d) + 1024;   // + static shared
  if (need <= smem_optin()) {
    static bool configured = false;
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(smem_optin() - 1024));
      if (e != cudaSuccess) return e;
      configured = true;
    }
    chol_inv_kernel<T><<<1, 1024, chol_smem_bytes<T>(d), st>>>(d, G, ldg, R, Rinv, ldr, info, shift_count,
                                                                 gate_out, gate_in, nullptr);
    note_launch();
  } else {
    if (gstore == nullptr) return cudaErrorInvalidValue;
    chol_inv_kernel<T><<<1, 1024, 0, st>>>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in,
                                            reinterpret_cast<T*>(gstore));
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace

size_t chol_global_bytes(int d, bool fp64) {
  size_t need = fp64 ? chol_smem_bytes<double>(d) : chol_smem_bytes<float>(d);
  return need + 1024 <= smem_optin() ? 0 : need;
}

cudaError_t chol_inv(int d, const float* G, int64_t ldg, float* R, float* Rinv, int64_t ldr, int* info,
                     double* shift_count, int* gate_out, const int* gate_in, void* gstore, bool fp64,
                     cudaStream_t st) {
  if (fp64)
    return launch_chol<double>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in, gstore, st);
  return launch_chol<float>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in, gstore, st);
}

cudaError_t transpose_small(int d, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t st) {
  int blocks = std::max(1, std::min(64, (d * d + 255) / 256));
  transpose_kernel<<<blocks, 256, 0, st>>>(d, X, ldx, Y, ldy);
  note_launch();
  return cudaGetLastError();
}

cudaError_t write_L(int d, const float* Rh, int64_t ldrh, float* L, int64_t ldl, double* l2,
                    cudaStream_t st) {
  int blocks = std::max(1, std::min(64, (d * d + 255) / 256));
  write_L_kernel<<<blocks, 256, 0, st>>>(d, Rh, ldrh, L, ldl, l2);
  note_launch();
  return cudaGetLastError();
}

cudaError_t init_scratch(int* info, int* gates, int ngates, double* scal, int nscal, cudaStream_t st) {
  init_kernel<<<1, 64, 0, st>>>(info, gates, ngates, scal, nscal);
  note_launch();
  return cudaGetLastError();
}

cudaError_t finish_diag(const double* scal, double* diag, int* info, cudaStream_t st) {
  finish_diag_kernel<<<1, 32, 0, st>>>(scal, diag, info);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_matrix(int64_t rows, int64_t cols, const float* X, int64_t ldx, float* Y, int64_t ldy,
                        cudaStream_t st) {
  int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 8);
  copy_kernel<<<blocks, 256, 0, st>>>(rows, cols, X, ldx, Y, ldy);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rqlp
