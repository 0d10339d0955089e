// Shared declarations of the Rand-QLP CUDA library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rqlp.h"

// Return the CUDA error of x from the enclosing function.
#define CK(x)                         \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

namespace rqlp {

// NVTX range over the enqueueing of one step of the chain (host side; a
// no-op unless a profiler attaches).
struct Range {
  explicit Range(const char* name);
  ~Range();
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Round x up to a multiple of a (a > 0); ceil(x / a).
__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int64_t cdiv(int64_t x, int64_t a) { return (x + a - 1) / a; }

// Bump allocator over the caller's workspace (256-byte aligned slices). A
// "dry" arena only measures, so sizing and use share one code path.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  bool dry = false;
  template <typename T>
  T* take(size_t count) {
    off = (size_t)round_up((int64_t)off, 256);
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

int sm_count();

// Asynchronous global -> shared copies (cp.async): `bytes` of the copy are
// read from src, the rest of the 4- or 16-byte destination is zero-filled
// (bytes == 0 reads nothing). The 16-byte form needs both addresses 16-byte
// aligned. Completion is tracked per thread in commit groups.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int bytes) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes = 16) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Cumulative count of kernels this library has launched in the process
// (reported by rqlp_kernel_launches). Every launch site calls note_launch().
void note_launch(int n = 1);

// Optional per-pass timing: when enabled, every pass over A is bracketed by a
// CUDA event pair recorded on the launching stream.
bool profiling_on();
void profile_mark_begin(cudaStream_t st);
void profile_mark_end(cudaStream_t st, int tag);

// ---------------------------------------------------------------- FP32 SIMT GEMM
// C[M x N] = op(A)[M x K] * B[K x N], op(A) = A^T when transA, row-major.
// splits > 1 uses `part` (splits * M * N floats) and a fixed-order reduction.
// sumsq (optional): += sum of squares of the A elements read.
// gate (optional) with gate_mode 1: *gate == 0 -> C = A (B taken as identity,
// needs !transA, K == N, one slice); gate_mode 2: *gate == 0 -> no work.
// b_upper: B is upper triangular (k-tiles beyond the column tile are skipped).
// lower_only (M == N, a Gram matrix whose reader takes its lower triangle):
// tiles whose entries all lie above the diagonal are skipped and C's strict
// upper triangle is left undefined.
enum GateMode { kGateNone = 0, kGateCopy = 1, kGateSkip = 2 };
cudaError_t gemm_f32_ex(bool transA, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc, int splits, float* part,
                        double* sumsq, const int* gate, int gate_mode, bool b_upper, cudaStream_t st,
                        bool lower_only = false);
int gemm_f32_splits(int64_t M, int64_t N, int64_t K);
size_t gemm_f32_part_floats(int64_t M, int64_t N, int64_t K);

// Grouped form for batches: one launch covers job b = 0..count-1, C_b =
// op(A_b) B_b, each with its own sizes, gate and options (no split-K).
// tile_start (device, count + 1 ints): exclusive prefix sum of the per-job
// tile counts cdiv(M, BM) * cdiv(N, BN) for the configuration's tile.
struct GroupGemm {
  const float* A; const float* B; float* C;
  int64_t lda, ldb, ldc;
  int64_t M, N, K;
  double* sumsq;
  const int* gate;
  int gate_mode;
  int b_upper;
  int lower_only;   // a Gram read by its lower triangle: tiles above the diagonal are skipped
};
// Tile shapes (kGroupCfgs) times grid modes: choice < kGroupCfgs is a
// persistent grid, choice - kGroupCfgs the same tile with one CTA per tile.
constexpr int kGroupCfgs = 6;
constexpr int kGroupChoices = 2 * kGroupCfgs;
void grouped_tile(int cfg, int* bm, int* bn);
cudaError_t gemm_grouped(bool transA, int choice, const GroupGemm* jobs, const int* tile_start, int count,
                         int total_tiles, cudaStream_t st);
// Runs every one-time query of the grouped kernels (call before capturing).
cudaError_t gemm_grouped_prepare();

// ---------------------------------------------------------------- d x d kernels
// R^T R = G (+ s I on breakdown; raises *gate_out), Rinv = R^{-1}; gate_in == 0
// -> R = Rinv = I. gstore: global scratch when the factor does not fit in
// shared memory (chol_global_bytes(d, fp64) bytes, else unused).
cudaError_t chol_inv(int d, const float* G, int64_t ldg, float* R, float* Rinv, int64_t ldr, int* info,
                     double* shift_count, int* gate_out, const int* gate_in, void* gstore, bool fp64,
                     cudaStream_t st);
size_t chol_global_bytes(int d, bool fp64);
// One CTA per job; every factor in shared memory (chol_batched_fits(dmax)).
struct CholJob {
  int d;
  const float* G; int64_t ldg;
  float* R; float* Rinv; int64_t ldr;
  int* info; double* shift_count; int* gate_out; const int* gate_in;
};
bool chol_batched_fits(int dmax, bool fp64);
cudaError_t chol_inv_batched(const CholJob* jobs, int count, int dmax, bool fp64, cudaStream_t st);
// count == 0 only configures the kernel (call before capturing).
// Batched small steps, one CTA per job.
struct SmallJob {
  int d;
  const float* X; int64_t ldx;   // transpose: source; write_L: Rhat
  float* Y; int64_t ldy;         // transpose: destination; write_L: L
  double* scal;                  // the job's scalars [||A||^2, ||L||^2, shifts, -]
  int* info;
  double* diag;                  // optional output (4 doubles)
  int* gates; int ngates;        // gate_clear / copy_gated: ngates = the gate's index
  int64_t rows;                  // copy_gated: rows of X and Y (d columns)
};
cudaError_t init_batched(const SmallJob* jobs, int count, cudaStream_t st);
cudaError_t transpose_batched(const SmallJob* jobs, int count, cudaStream_t st);
cudaError_t write_L_batched(const SmallJob* jobs, int count, cudaStream_t st);
cudaError_t finish_diag_batched(const SmallJob* jobs, int count, cudaStream_t st);
// gates[ngates] = 0 for every job; Y = X (rows x d) for the jobs whose gates[ngates] is raised.
cudaError_t gate_clear_batched(const SmallJob* jobs, int count, cudaStream_t st);
cudaError_t copy_gated_batched(const SmallJob* jobs, int count, cudaStream_t st);
cudaError_t transpose_small(int d, const float* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t st);
cudaError_t write_L(int d, const float* Rh, int64_t ldrh, float* L, int64_t ldl, double* l2_accum,
                    cudaStream_t st);
cudaError_t init_scratch(int* info, int* gates, int ngates, double* scal, int nscal, cudaStream_t st);
cudaError_t finish_diag(const double* scal, double* diag, int* info, cudaStream_t st);
// Y += X (rows x cols).
cudaError_t add_matrix(int64_t rows, int64_t cols, const float* X, int64_t ldx, float* Y, int64_t ldy,
                       cudaStream_t st);
// gate (optional): *gate == 0 -> no copy.
cudaError_t copy_matrix(int64_t rows, int64_t cols, const float* X, int64_t ldx, float* Y, int64_t ldy,
                        cudaStream_t st, const int* gate = nullptr);

// ---------------------------------------------------------------- sparse A (CSR, device arrays)
struct SparseA {
  int64_t m, n, nnz;
  const int64_t* row_ptr;   // m + 1
  const int* col_idx;       // nnz
  const float* vals;        // nnz
};
// Device bytes for A's transpose in CSR form (built by sparse_build_csc).
size_t sparse_csc_bytes(int64_t n, int64_t nnz);
cudaError_t sparse_build_csc(const SparseA& a, void* ws, SparseA* t, int* info, cudaStream_t st);
// Y (s.m x d) = S X (X s.n x d); sumsq += sum of S's squared values (optional).
cudaError_t sparse_spmm(const SparseA& s, const float* X, int64_t ldx, int d, float* Y, int64_t ldy, double* sumsq,
                        int* info, cudaStream_t st);

// ---------------------------------------------------------------- learned (q, p)
size_t mlp_workspace_floats(int batch);
cudaError_t mlp_forward(const float* prm, const float* X, int batch, float* est, cudaStream_t st);
cudaError_t mlp_grad(const float* prm, const float* X, const float* Y, int batch, float* grad, float* loss,
                     void* ws, cudaStream_t st);
cudaError_t mlp_adam(float* prm, const float* g, float* m1, float* m2, int n, float lr, float beta1, float beta2,
                     float eps, int step, cudaStream_t st);
cudaError_t probe_features(const float* R, int64_t ldr, int w, int k, int64_t mn, float* feat, cudaStream_t st);
cudaError_t predict_qp(const float* est, const float* prm, const int* info, double target, int k, int* qp,
                       cudaStream_t st);

}  // namespace rqlp
