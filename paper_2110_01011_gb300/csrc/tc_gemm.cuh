// Tensor-core (tcgen05 / TMEM / TMA) passes over A in BF16 split precision.
#pragma once

#include "common.cuh"

namespace rqlp {

// True when the BF16x3 passes can run on the current device (sm_103 with the
// tensor-map encoder available).
bool tc_supported(const float* A, int64_t lda, const float* Omega, int64_t ldo);

// Workspace and launch state of the BF16x3 passes of one factorisation: the
// BF16 halves of A (written once, by the first pass), the BF16 halves of the
// current X (transposed, K-major), and the stream-K partial tiles.
class TcEngine {
 public:
  void layout(Arena& ar, int64_t m, int64_t n, int d);
  void reset() { split_of_ = nullptr; }
  // transA: out (n x d) = A^T X (X m x d); else out (m x d) = A X (X n x d).
  // sumsq (only with the pass that splits A) receives ||A||_F^2.
  cudaError_t pass(bool transA, const float* A, int64_t m, int64_t n, int64_t lda, const float* X, int64_t ldx,
                   int d, float* out, int64_t ldout, double* sumsq, int* info, cudaStream_t st);

 private:
  int64_t m_ = 0, n_ = 0, ldb_ = 0, ldk_ = 0;
  int d_ = 0, npad_ = 0, G_ = 0;
  uint16_t *Ahi_ = nullptr, *Alo_ = nullptr, *Xhi_ = nullptr, *Xlo_ = nullptr;
  float* part_ = nullptr;
  int* flag_ = nullptr;
  int* cnt_ = nullptr;
  const float* split_of_ = nullptr;
};

}  // namespace rqlp
