// Tensor-core (tcgen05 / TMEM / TMA) passes over A in BF16 split precision.
#pragma once

#include "common.cuh"

namespace rqlp {

// True when the BF16x3 passes can run on the current device (sm_103 with the
// tensor-map encoder available).
bool tc_supported(const float* A, int64_t lda, const float* Omega, int64_t ldo);

// Workspace and launch state of BF16x3 tensor-core products over one split
// operand: the BF16 halves of a matrix A (rows x cols, written by split()),
// the BF16 halves of the current X operand (transposed, K-major), and the
// partial tiles of stream-K / of the Gram reduction. Capacities are fixed by
// layout(); split() must be called again whenever A's contents change.
class TcEngine {
 public:
  // rows_cap x cols_cap: largest split A; d_cap: largest output width; k_cap:
  // largest K of a pass (rows of X); gram: reserve the Gram partial slots;
  // three_part: also keep A_lo2 = bf16(A - A_hi - A_lo) and X_lo2 (exact mode).
  void layout(Arena& ar, int64_t rows_cap, int64_t cols_cap, int d_cap, int64_t k_cap, bool gram,
              bool three_part = false);
  void reset() { split_of_ = nullptr; }
  // Bracket this engine's MMA kernel with the library's profiling events.
  void set_profiled(bool on) { profiled_ = on; }
  // A (rows x cols FP32) -> A_hi, A_lo; sumsq (optional) += ||A||_F^2.
  cudaError_t split(const float* A, int64_t rows, int64_t cols, int64_t lda, double* sumsq, cudaStream_t st);
  // transA: out (cols x d) = A^T X (X rows x d); else out (rows x d) = A X
  // (X cols x d). Splits A first unless it is the current split. exact: A and
  // X in three parts, six products (needs three_part).
  cudaError_t pass(bool transA, const float* A, int64_t rows, int64_t cols, int64_t lda, const float* X,
                   int64_t ldx, int d, float* out, int64_t ldout, double* sumsq, int* info, cudaStream_t st,
                   bool exact = false);
  // G (cols x cols, ldg) = A^T A of the current split (cols <= 256).
  cudaError_t gram(float* G, int64_t ldg, int* info, cudaStream_t st);

 private:
  int64_t rows_cap_ = 0, cols_cap_ = 0, k_cap_ = 0, ldb_ = 0;
  int d_cap_ = 0, G_ = 0;
  int64_t m_ = 0, n_ = 0;   // dims of the current split
  uint16_t *Ahi_ = nullptr, *Alo_ = nullptr, *Alo2_ = nullptr, *Xhi_ = nullptr, *Xlo_ = nullptr, *Xlo2_ = nullptr;
  float* part_ = nullptr;
  float* gpart_ = nullptr;
  int* flag_ = nullptr;
  int* cnt_ = nullptr;
  const float* split_of_ = nullptr;
  bool profiled_ = false;
};

}  // namespace rqlp
