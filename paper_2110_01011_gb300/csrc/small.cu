// Small kernels of the chain: the d x d transpose, the L write-out with
// ||L||_F^2, scratch initialisation, the diagnostics word and a strided copy.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rqlp {

namespace {

__device__ void post_error(int* info, int code, int detail) {
  if (info != nullptr && atomicCAS(info, 0, code) == 0) info[1] = detail;
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
// ||L||_F^2 accumulated into *l2 (double, one atomic per CTA).
__global__ void write_L_kernel(int d, const float* __restrict__ Rh, int64_t ldrh, float* __restrict__ L,
                               int64_t ldl, double* l2) {
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
  if (threadIdx.x == 0 && l2 != nullptr) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(l2, s);
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
                            float* __restrict__ Y, int64_t ldy, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / cols, c = e % cols;
    Y[r * ldy + c] = X[r * ldx + c];
  }
}

// ---- batched forms: blockIdx.x = job
__global__ void init_batched_kernel(const SmallJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x;
  if (b >= count) return;
  const SmallJob& j = jobs[b];
  const int t = threadIdx.x;
  if (t < 2) j.info[t] = 0;
  if (t < j.ngates) j.gates[t] = 0;
  if (t < 4) j.scal[t] = 0.0;
}

__global__ void transpose_batched_kernel(const SmallJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x;
  if (b >= count) return;
  const SmallJob& j = jobs[b];
  for (int e = threadIdx.x; e < j.d * j.d; e += blockDim.x) {
    const int i = e / j.d, l = e % j.d;
    j.Y[(int64_t)l * j.ldy + i] = j.X[(int64_t)i * j.ldx + l];
  }
}

__global__ void write_L_batched_kernel(const SmallJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x;
  if (b >= count) return;
  const SmallJob& j = jobs[b];
  __shared__ double red[32];
  double acc = 0.0;
  for (int e = threadIdx.x; e < j.d * j.d; e += blockDim.x) {
    const int i = e / j.d, c = e % j.d;
    const float v = c <= i ? j.X[(int64_t)c * j.ldx + i] : 0.f;
    j.Y[(int64_t)i * j.ldy + c] = v;
    acc += (double)v * (double)v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    j.scal[1] = s;
  }
}

__global__ void finish_diag_batched_kernel(const SmallJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const SmallJob& j = jobs[b];
  const double a2 = j.scal[0], l2 = j.scal[1];
  if (!isfinite(a2)) post_error(j.info, RQLP_ERR_NONFINITE, 0);
  if (j.diag != nullptr) {
    j.diag[0] = a2;
    j.diag[1] = l2;
    j.diag[2] = a2 - l2;
    j.diag[3] = j.scal[2];
  }
}

}  // namespace

cudaError_t init_batched(const SmallJob* jobs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  init_batched_kernel<<<count, 32, 0, st>>>(jobs, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t transpose_batched(const SmallJob* jobs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  transpose_batched_kernel<<<count, 256, 0, st>>>(jobs, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t write_L_batched(const SmallJob* jobs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  write_L_batched_kernel<<<count, 256, 0, st>>>(jobs, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t finish_diag_batched(const SmallJob* jobs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  finish_diag_batched_kernel<<<(count + 127) / 128, 128, 0, st>>>(jobs, count);
  note_launch();
  return cudaGetLastError();
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

__global__ void gate_clear_batched_kernel(const SmallJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < count) jobs[b].gates[jobs[b].ngates] = 0;
}

// blockIdx.y = job; the job's rows x d elements over blockIdx.x.
__global__ void copy_gated_batched_kernel(const SmallJob* __restrict__ jobs) {
  const SmallJob& j = jobs[blockIdx.y];
  if (j.gates[j.ngates] == 0) return;
  const int64_t total = j.rows * j.d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / j.d, c = e % j.d;
    j.Y[r * j.ldy + c] = j.X[r * j.ldx + c];
  }
}

cudaError_t gate_clear_batched(const SmallJob* jobs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  gate_clear_batched_kernel<<<(count + 127) / 128, 128, 0, st>>>(jobs, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_gated_batched(const SmallJob* jobs, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (count > 65535) return cudaErrorInvalidValue;   // one grid row per job
  copy_gated_batched_kernel<<<dim3(16, count), 256, 0, st>>>(jobs);
  note_launch();
  return cudaGetLastError();
}

__global__ void add_kernel(int64_t rows, int64_t cols, const float* __restrict__ X, int64_t ldx,
                           float* __restrict__ Y, int64_t ldy) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    Y[r * ldy + c] += X[r * ldx + c];
  }
}

cudaError_t add_matrix(int64_t rows, int64_t cols, const float* X, int64_t ldx, float* Y, int64_t ldy,
                       cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 8);
  add_kernel<<<blocks, 256, 0, st>>>(rows, cols, X, ldx, Y, ldy);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_matrix(int64_t rows, int64_t cols, const float* X, int64_t ldx, float* Y, int64_t ldy,
                        cudaStream_t st, const int* gate) {
  int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 8);
  copy_kernel<<<blocks, 256, 0, st>>>(rows, cols, X, ldx, Y, ldy, gate);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rqlp
