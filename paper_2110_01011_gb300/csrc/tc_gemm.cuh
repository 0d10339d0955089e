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
  // Split A by row blocks as they arrive: begin_split names A (rows x cols,
  // device, whose rows the caller fills) as the current split and resets the
  // tile counters; split_rows splits rows row0 .. row0 + rows - 1 (Ablock
  // points at row row0, lda); sumsq += their squares.
  cudaError_t begin_split(const float* A, int64_t rows, int64_t cols, cudaStream_t st);
  cudaError_t split_rows(const float* Ablock, int64_t row0, int64_t rows, int64_t lda, double* sumsq,
                         cudaStream_t st);
  // out = op(A_cur) X over K rows k0 .. k0 + K - 1 of the current split
  // (transA only for k0 > 0; X holds those K rows). Without transA, Mrows >= 0
  // restricts the product to A's rows m0 .. m0 + Mrows - 1 (out row 0 = row m0).
  cudaError_t pass_k(bool transA, int64_t k0, int64_t K, const float* X, int64_t ldx, int d, float* out,
                     int64_t ldout, int* info, cudaStream_t st, bool exact = false, int64_t m0 = 0,
                     int64_t Mrows = -1);
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

// ---------------------------------------------------------------- grouped passes (batched form)
// One problem's pass in a grouped launch: out (M x d) = op(A) X with the
// problem's tensor maps (CUtensorMap, in device memory): A_hi, A_lo over the
// panel layout (box {64, 32, 2} for op(A) = A^T, {32, 128, 1} for A) and
// X_hi^T, X_lo^T (box {32, npad}).
struct TcGJob {
  const void* mAhi;
  const void* mAlo;
  const void* mXhi;
  const void* mXlo;
  const void* mAlo2;        // three-part launches: A_lo2, X_lo2 (else unused)
  const void* mXlo2;
  float* out;
  long long ldo;
  int M, d, npad, kblocks, vec_out;
  uint32_t idesc;
  const int* xlo_nonzero;   // raised by prep_grouped when X has a low part
};
struct SplitJob {           // A (m x n) -> panels of A_hi, A_lo; sumsq += ||A||_F^2
  const float* A;
  long long lda, m, n, npan;
  void* hi;
  void* lo;
  void* lo2;                // bf16(A - A_hi - A_lo), or null (two parts)
  double* sumsq;
  int vec;                  // A 16-byte aligned with lda % 4 == 0
};
struct PrepJob {            // X (K x d) -> X_hi^T, X_lo^T (d x ldk)
  const float* X;
  long long ldx, K;
  int d;
  void* th;
  void* tl;
  void* tl2;                // bf16(X - X_hi - X_lo)^T, or null (two parts)
  long long ldk;
  int* flag;
};
constexpr size_t kTcMapBytes = 128;   // sizeof(CUtensorMap)
int tc_split_blocks(long long m, long long n);
int tc_prep_blocks(long long K, int d);
// start: count + 1 block prefix sums (tc_split_blocks / tc_prep_blocks).
cudaError_t split_grouped(const SplitJob* jobs, const int* start, int count, int total_blocks, cudaStream_t st);
cudaError_t prep_grouped(const PrepJob* jobs, const int* start, int count, int total_blocks, cudaStream_t st);
// units: (job, 128-row tile) pairs; CTA c takes units cta_start[c] .. cta_start[c + 1] - 1.
// G = 0 only configures the kernel (call before capturing).
// stall != 0 (fault-injection tests): CTA 0 withholds its first stage's loads,
// its bounded waits run out and `info` receives RQLP_ERR_TIMEOUT. exact: A and
// X in three parts, six products (every job's third-part maps are set).
cudaError_t tc_grouped_pass(bool transA, const TcGJob* jobs, const int2* units, const int* cta_start, int G,
                            int npad_max, int* info, int stall, bool exact, cudaStream_t st);
// Host encoders of the tensor maps above (false when the encoder is missing
// or rejects the arguments).
bool tc_panel_map(void* map, const void* base, long long m, long long panels, int bi, int bo, int bp, bool sw128);
bool tc_map2d(void* map, const void* base, long long inner, long long outer, long long pitch, int bi, int bo,
              bool sw128);
int tc_npad(int d);
uint32_t tc_idesc(int npad, bool a_mn_major);   // tcgen05.mma kind::f16, M = 128, BF16 in, FP32 accumulate

}  // namespace rqlp
