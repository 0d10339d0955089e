// Rand-QLP of a sparse A (CSR): the passes over A as sparse-times-dense
// products, the rest of the chain unchanged (section 5.1 factors sparse test
// matrices; Algorithm 1 only multiplies by A and A^T).
//
// A X: one warp per row of A, the lanes over the d columns of X (up to 8
// per lane), the row's nonzeros in order, FP32 accumulation. A^T X: the same
// kernel on A's transpose in CSR form (CSC of A), built on the device at the
// start of every factorisation: column counts, an exclusive scan, a scatter
// and a sort of each column's entries by row, so that every sum runs in a
// fixed order (the results are deterministic). Indices are checked on the
// device: a column index outside [0, n) or a row pointer that decreases
// reports RQLP_ERR_ARG in the status word and the bad entry is skipped.
#include <algorithm>

#include "common.cuh"

namespace rqlp {
namespace {

constexpr int kMaxPerLane = (RQLP_MAX_D + 31) / 32;

__device__ void post_arg_error(int* info) {
  if (info != nullptr && atomicCAS(info, 0, RQLP_ERR_ARG) == 0) info[1] = 0;
}

// Y (rows x d) = S X for S in CSR (rows x K), X (K x d, ldx); sumsq
// (optional): += sum of the squares of S's values.
__global__ void __launch_bounds__(256)
csr_spmm_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ val,
                int64_t rows, int64_t K, const float* __restrict__ X, int64_t ldx, int d, float* __restrict__ Y,
                int64_t ldy, double* sumsq, int* info) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double sq = 0.0;
  for (int64_t r = warp; r < rows; r += nwarps) {
    float acc[kMaxPerLane];
#pragma unroll
    for (int t = 0; t < kMaxPerLane; ++t) acc[t] = 0.f;
    const int64_t s = ptr[r], e = ptr[r + 1];
    if (e < s) {
      if (lane == 0) post_arg_error(info);
      continue;
    }
    for (int64_t p = s; p < e; ++p) {
      const int j = idx[p];
      const float v = val[p];
      if (j < 0 || j >= K) {
        if (lane == 0) post_arg_error(info);
        continue;
      }
      if (sumsq != nullptr && lane == 0) sq += (double)v * (double)v;
      const float* x = X + (int64_t)j * ldx;
#pragma unroll
      for (int t = 0; t < kMaxPerLane; ++t) {
        const int c = lane + 32 * t;
        if (c < d) acc[t] = fmaf(v, x[c], acc[t]);
      }
    }
    float* y = Y + r * ldy;
#pragma unroll
    for (int t = 0; t < kMaxPerLane; ++t) {
      const int c = lane + 32 * t;
      if (c < d) y[c] = acc[t];
    }
  }
  if (sumsq != nullptr && lane == 0 && sq != 0.0) atomicAdd(sumsq, sq);
}

// counts[j] = number of entries in column j (valid indices only).
__global__ void csc_count_kernel(const int* __restrict__ idx, int64_t nnz, int64_t n, int* __restrict__ counts) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
    const int j = idx[p];
    if (j >= 0 && j < n) atomicAdd(&counts[j], 1);
  }
}

// col_ptr = exclusive prefix sum of counts (n + 1 entries); one CTA.
__global__ void __launch_bounds__(1024) csc_scan_kernel(const int* __restrict__ counts, int64_t n,
                                                        int64_t* __restrict__ col_ptr) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = (int64_t)t * chunk, e = std::min<int64_t>(n, b + chunk);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const int64_t v = part[i];
      part[i] = run;
      run += v;
    }
    col_ptr[n] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t i = b; i < e; ++i) {
    col_ptr[i] = run;
    run += counts[i];
  }
}

// Scatter every entry (r, j, v) to column j's segment (fill: n zeroed ints).
__global__ void __launch_bounds__(256)
csc_fill_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ val,
                int64_t rows, int64_t n, const int64_t* __restrict__ col_ptr, int* __restrict__ fill,
                int* __restrict__ ridx, float* __restrict__ rval) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    const int64_t s = ptr[r], e = ptr[r + 1];
    for (int64_t p = s + lane; p < e; p += 32) {
      const int j = idx[p];
      if (j < 0 || j >= n) continue;
      const int64_t pos = col_ptr[j] + atomicAdd(&fill[j], 1);
      ridx[pos] = (int)r;
      rval[pos] = val[p];
    }
  }
}

// Each column's entries in increasing row order (insertion sort, a thread
// per column): the scatter's order depends on the atomics.
__global__ void csc_sort_kernel(const int64_t* __restrict__ col_ptr, int64_t n, int* __restrict__ ridx,
                                float* __restrict__ rval) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = col_ptr[j], e = col_ptr[j + 1];
    for (int64_t p = s + 1; p < e; ++p) {
      const int r = ridx[p];
      const float v = rval[p];
      int64_t q = p - 1;
      while (q >= s && ridx[q] > r) {
        ridx[q + 1] = ridx[q];
        rval[q + 1] = rval[q];
        --q;
      }
      ridx[q + 1] = r;
      rval[q + 1] = v;
    }
  }
}

int spmm_blocks(int64_t rows) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(rows, 8), (int64_t)sm_count() * 16));
}

}  // namespace

size_t sparse_csc_bytes(int64_t n, int64_t nnz) {
  Arena ar;
  ar.dry = true;
  ar.take<int64_t>((size_t)n + 1);
  ar.take<int>((size_t)nnz);
  ar.take<float>((size_t)nnz);
  ar.take<int>((size_t)n);
  return ar.off;
}

cudaError_t sparse_build_csc(const SparseA& a, void* ws, SparseA* t, int* info, cudaStream_t st) {
  Arena ar;
  ar.base = static_cast<char*>(ws);
  ar.cap = sparse_csc_bytes(a.n, a.nnz);
  int64_t* col_ptr = ar.take<int64_t>((size_t)a.n + 1);
  int* ridx = ar.take<int>((size_t)a.nnz);
  float* rval = ar.take<float>((size_t)a.nnz);
  int* counts = ar.take<int>((size_t)a.n);
  CK(cudaMemsetAsync(counts, 0, sizeof(int) * a.n, st));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(a.nnz, 256), (int64_t)sm_count() * 8));
  if (a.nnz > 0) {
    csc_count_kernel<<<blocks, 256, 0, st>>>(a.col_idx, a.nnz, a.n, counts);
    note_launch();
  }
  csc_scan_kernel<<<1, 1024, 0, st>>>(counts, a.n, col_ptr);
  CK(cudaMemsetAsync(counts, 0, sizeof(int) * a.n, st));   // reused as the fill cursor
  csc_fill_kernel<<<spmm_blocks(a.m), 256, 0, st>>>(a.row_ptr, a.col_idx, a.vals, a.m, a.n, col_ptr, counts, ridx,
                                                    rval);
  csc_sort_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>(cdiv(a.n, 128), (int64_t)sm_count() * 4)), 128, 0,
                    st>>>(col_ptr, a.n, ridx, rval);
  note_launch(3);
  t->m = a.n;
  t->n = a.m;
  t->nnz = a.nnz;
  t->row_ptr = col_ptr;
  t->col_idx = ridx;
  t->vals = rval;
  (void)info;
  return cudaGetLastError();
}

cudaError_t sparse_spmm(const SparseA& s, const float* X, int64_t ldx, int d, float* Y, int64_t ldy, double* sumsq,
                        int* info, cudaStream_t st) {
  if (d > RQLP_MAX_D) return cudaErrorInvalidValue;
  csr_spmm_kernel<<<spmm_blocks(s.m), 256, 0, st>>>(s.row_ptr, s.col_idx, s.vals, s.m, s.n, X, ldx, d, Y, ldy, sumsq,
                                                    info);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rqlp
