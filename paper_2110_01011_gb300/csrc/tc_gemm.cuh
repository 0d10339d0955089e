// Tensor-core (tcgen05 / TMEM) passes over A in BF16 split precision.
#pragma once

#include "common.cuh"

namespace rqlp {

// True when the BF16x3 passes can run on these operands (device, layout).
bool tc_supported(const float* A, int64_t lda, const float* Omega, int64_t ldo);

// Workspace and launch state of the BF16x3 passes of one factorisation.
struct TcEngine {
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void layout(Arena& ar, int64_t m, int64_t n, int d);
  // transA: Y (n x d) = A^T X (X m x d); else Z (m x d) = A X (X n x d).
  cudaError_t pass(bool transA, const float* A, int64_t m, int64_t n, int64_t lda, const float* X,
                   int64_t ldx, int d, float* out, int64_t ldout, double* sumsq, cudaStream_t st);
};

}  // namespace rqlp
