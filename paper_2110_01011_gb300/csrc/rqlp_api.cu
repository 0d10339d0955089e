// C ABI of the Rand-QLP library and the stream-ordered plan that runs the
// truncated chain (section 3.1, Algorithm 1, with d = k + p sketch columns
// and q power passes):
//
//   Y = A^T Omega -> P~ = qf(Y) -> q x [Z = qf(A P~), P~ = qf(A^T Z)]
//   -> (Q, R) = qr(A P~) -> (P^, R^) = qr(R^T), L = R^^T, P = P~ P^.
//
// qf is CholeskyQR on the GPU. Intermediate bases (inside the power passes)
// take one CholeskyQR pass: any upper-triangular right factor keeps
// qf((A^T A)^q A^T Omega) unchanged, so they only need to stay well
// conditioned. The bases that enter the result (the last P~, Q, and the QR
// of R^T) take CholeskyQR2, plus a third pass when a Cholesky had to be
// shifted (shifted CholeskyQR3); that pass is gated on a device flag so the
// launch sequence is static and capturable.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace rqlp {
namespace {

constexpr int kGates = 8;   // gate words: one per final orthonormalisation, [3] intermediate ones
constexpr int kInterGate = 3;
constexpr int kScal = 4;    // [0] ||A||^2, [1] ||L||^2, [2] shifted Cholesky count, [3] spare

// Building blocks of the chain for a fixed sketch width d, with their scratch.
class Ops {
 public:
  Ops(int d, const rqlp_opts& o) : d_(d), dcap_(d), ld_(round_up(d, 4)), o_(o) {}

  // Three BF16 parts per pass operand (six products) instead of two.
  void set_three_part(bool on) { three_ = on; }
  // Sparse A (CSR) and its transpose: the passes become sparse products.
  void set_sparse(const SparseA* a, const SparseA* at) {
    sp_ = a;
    spt_ = at;
  }

  // part_floats: largest split-K partial buffer any product of the caller needs.
  void layout(Arena& ar, size_t part_floats, bool with_tc, int64_t m, int64_t n) {
    const int64_t dd = (int64_t)dcap_ * ld_;
    G_ = ar.take<float>(dd);
    for (int i = 0; i < 3; ++i) {
      R_[i] = ar.take<float>(dd);
      Ri_[i] = ar.take<float>(dd);
    }
    Ra_ = ar.take<float>(dd);
    part_ = ar.take<float>(std::max<size_t>(part_floats, 1));
    scal = ar.take<double>(kScal);
    gates = ar.take<int>(kGates);
    cstore_ = ar.take<char>(chol_global_bytes(dcap_, o_.small_fp64 != 0));
    if (with_tc) {
      tc_.layout(ar, m, n, dcap_, std::max(m, n), false, three_);
      tc_.set_profiled(true);
      // Tall d-column operands of CholeskyQR: the Gram (BF16x3) and the
      // products X R^{-1} (exact mode, six products) on the tensor cores.
      tcs_.layout(ar, std::max(m, n), dcap_, dcap_, dcap_, true, /*three_part=*/true);
    }
    tc_on_ = with_tc;
  }
  void bind(cudaStream_t st, int* info) { st_ = st; info_ = info; }
  int64_t ld() const { return ld_; }
  // Current sketch width (<= the capacity the workspace was laid out for).
  void set_d(int d) { d_ = d; }
  int d() const { return d_; }
  const float* R(int slot) const { return R_[slot]; }
  // R factor of X (rows x d) in slot 0 without forming X R^{-1} (the probe).
  // The Gram is FP32 in both precisions: the probe's small R-diagonal entries
  // carry the Gram's error amplified by kappa(X)^2, and they are the features.
  // gates[0] is raised if the Cholesky had to shift.
  cudaError_t gram_chol(const float* X, int64_t ldx, int64_t rows) {
    CK(gram(X, ldx, rows, nullptr));
    return chol(0, &gates[0], nullptr, true);
  }
  // out = X R0^{-1} with the inverse already in slot 0. For a prefix of the
  // columns the leading block of the triangular inverse is the inverse of the
  // leading block, so a probe of a wider sketch serves every narrower width.
  cudaError_t apply_r0(const float* X, int64_t ldx, int64_t rows, float* out, int64_t ldout) {
    if (tc_on_ && rows > (int64_t)d_) {
      tcs_.reset();
      CK(tcs_.split(X, rows, d_, ldx, nullptr, st_));
      return tcs_.pass(false, X, rows, d_, ldx, Ri_[0], ld_, d_, out, ldout, nullptr, info_, st_, true);
    }
    return trmm(X, ldx, rows, Ri_[0], out, ldout, nullptr);
  }

  cudaError_t init() {
    tc_.reset();
    tcs_.reset();
    return init_scratch(info_, gates, kGates, scal, kScal, st_);
  }

  // transA: out (n x d) = A^T X (X m x d); else out (m x d) = A X (X n x d).
  cudaError_t pass(bool transA, const float* A, int64_t m, int64_t n, int64_t lda, const float* X,
                   int64_t ldx, float* out, int64_t ldout, double* sumsq) {
    if (sp_ != nullptr) {
      const bool prof = profiling_on();
      if (prof) profile_mark_begin(st_);
      cudaError_t e = sparse_spmm(transA ? *spt_ : *sp_, X, ldx, d_, out, ldout, sumsq, info_, st_);
      if (prof) profile_mark_end(st_, transA ? 1 : 0);
      return e;
    }
    if (o_.precision == RQLP_PREC_BF16X3)   // the engine brackets its MMA kernel when profiling
      return tc_.pass(transA, A, m, n, lda, X, ldx, d_, out, ldout, sumsq, info_, st_, three_);
    const bool prof = profiling_on();
    if (prof) profile_mark_begin(st_);
    const int64_t M = transA ? n : m, K = transA ? m : n;
    cudaError_t e = gemm_f32_ex(transA, M, d_, K, A, lda, X, ldx, out, ldout, gemm_f32_splits(M, d_, K), part_,
                                sumsq, nullptr, kGateNone, false, st_);
    if (prof) profile_mark_end(st_, transA ? 1 : 0);
    return e;
  }
  // out (n x d) = A(r0 .. r0 + rows - 1, :)^T X (X: those rows), A m x n on
  // the device; first: rows start at 0 (the split of A begins). ||A||_F^2 of
  // the rows rides along into scal[0].
  cudaError_t pass_rows(const float* A, int64_t m, int64_t n, int64_t lda, int64_t r0, int64_t rows,
                        const float* X, int64_t ldx, float* out, int64_t ldout) {
    if (o_.precision == RQLP_PREC_BF16X3) {
      if (r0 == 0) CK(tc_.begin_split(A, m, n, st_));
      CK(tc_.split_rows(A + r0 * lda, r0, rows, lda, &scal[0], st_));
      return tc_.pass_k(true, r0, rows, X, ldx, d_, out, ldout, info_, st_, three_);
    }
    const bool prof = profiling_on();
    if (prof) profile_mark_begin(st_);
    cudaError_t e = gemm_f32_ex(true, n, d_, rows, A + r0 * lda, lda, X, ldx, out, ldout,
                                gemm_f32_splits(n, d_, rows), part_, &scal[0], nullptr, kGateNone, false, st_);
    if (prof) profile_mark_end(st_, 1);
    return e;
  }
  // Y (n x d) = A^T (A X) by row panels of A: Z_b = A_b X, then Y += A_b^T Z_b
  // while A_b is still in L2 (panels of at most ~48 MB of A's pass operands).
  // Z (m x d, ld_) receives A X, T (n x d, ld_) is scratch. Z is not
  // orthonormalised: R(A^T A X) = R(A^T qf(A X)), and any triangular right
  // factor leaves the qf of the product unchanged (reading C3).
  cudaError_t power_fused(const float* A, int64_t m, int64_t n, int64_t lda, const float* X, int64_t ldx, float* Y,
                          int64_t ldy, float* Z, float* T) {
    const bool tc = o_.precision == RQLP_PREC_BF16X3;
    const int64_t h = fused_rows(m, n, tc ? (three_ ? 6 : 4) : 4);
    for (int64_t r0 = 0; r0 < m; r0 += h) {   // (in the BF16x3 form A's split is current: the sketch made it)
      const int64_t rows = std::min(h, m - r0);
      float* zb = Z + r0 * ld_;
      float* dst = r0 == 0 ? Y : T;
      const int64_t ldd = r0 == 0 ? ldy : ld_;
      if (tc) {
        CK(tc_.pass_k(false, 0, n, X, ldx, d_, zb, ld_, info_, st_, three_, r0, rows));
        CK(tc_.pass_k(true, r0, rows, zb, ld_, d_, dst, ldd, info_, st_, three_));
      } else {
        CK(gemm_f32_ex(false, rows, d_, n, A + r0 * lda, lda, X, ldx, zb, ld_, gemm_f32_splits(rows, d_, n), part_,
                       nullptr, nullptr, kGateNone, false, st_));
        CK(gemm_f32_ex(true, n, d_, rows, A + r0 * lda, lda, zb, ld_, dst, ldd, gemm_f32_splits(n, d_, rows), part_,
                       nullptr, nullptr, kGateNone, false, st_));
      }
      if (r0 > 0) CK(add_matrix(n, d_, T, ld_, Y, ldy, st_));
    }
    return cudaSuccess;
  }
  // Row-panel height of power_fused: at most ~48 MB of A's pass operands
  // (bpe bytes per element of A), a multiple of 128 rows.
  static int64_t fused_rows(int64_t m, int64_t n, int64_t bpe) {
    return std::min<int64_t>(m, std::max<int64_t>(128, (48ll << 20) / (n * bpe) / 128 * 128));
  }
  // Largest split-K partial buffer of power_fused in the FP32 form: a panel's
  // A_b X has fewer rows than A X, so it may take more K slices.
  static size_t fused_part_floats(int64_t m, int64_t n, int d) {
    const int64_t h = fused_rows(m, n, 4), tail = m % h;
    size_t p = std::max(gemm_f32_part_floats(h, d, n), gemm_f32_part_floats(n, d, h));
    if (tail > 0) p = std::max({p, gemm_f32_part_floats(tail, d, n), gemm_f32_part_floats(n, d, tail)});
    return p;
  }
  static size_t pass_part_floats(int64_t m, int64_t n, int d) {
    return std::max(gemm_f32_part_floats(n, d, m), gemm_f32_part_floats(m, d, n));
  }
  static size_t orth_part_floats(int64_t rows, int d) { return gemm_f32_part_floats(d, d, rows); }

  // G = X^T X, lower triangle (the Cholesky kernel reads G(i, j) for j <= i).
  cudaError_t gram(const float* X, int64_t ldx, int64_t rows, const int* gate) {
    return gemm_f32_ex(true, d_, d_, rows, X, ldx, X, ldx, G_, ld_, gemm_f32_splits(d_, d_, rows), part_,
                       nullptr, gate, kGateSkip, false, st_, /*lower_only=*/true);
  }
  // out = X Rinv (Rinv upper triangular); gate == 0 -> out = X.
  cudaError_t trmm(const float* X, int64_t ldx, int64_t rows, const float* Rinv, float* out, int64_t ldout,
                   const int* gate) {
    return gemm_f32_ex(false, rows, d_, d_, X, ldx, Rinv, ld_, out, ldout, 1, nullptr, nullptr, gate,
                       gate ? kGateCopy : kGateNone, true, st_);
  }
  // want_r: also write R (slot) besides R^{-1}; the passes that only
  // orthonormalise need the inverse alone.
  cudaError_t chol(int slot, int* gate_out, const int* gate_in, bool want_r) {
    return chol_inv(d_, G_, ld_, want_r ? R_[slot] : nullptr, Ri_[slot], ld_, info_, &scal[2], gate_out, gate_in,
                    cstore_, o_.small_fp64 != 0, st_);
  }
  // One CholeskyQR pass (shifted on breakdown) on the tensor cores: out =
  // X R^{-1}; gate_out raised if the Cholesky shifted. R only has to
  // precondition, so the BF16x3 Gram's rounding leaves the span of the result
  // untouched. X R^{-1} takes the exact mode: in BF16x3 its error, relative to
  // |X| |R^{-1}|, would be about kappa(X) times the result (measured: 1.6x the
  // leading-diagonal error of L on the 20000^2 class); six products bring it
  // to the FP32 product's level.
  cudaError_t tc_cqr(const float* X, int64_t ldx, int64_t rows, float* out, int64_t ldout, int slot,
                     int* gate_out, bool want_r) {
    tcs_.reset();
    CK(tcs_.split(X, rows, d_, ldx, nullptr, st_));
    CK(tcs_.gram(G_, ld_, info_, st_));
    CK(chol(slot, gate_out, nullptr, want_r));
    return tcs_.pass(false, X, rows, d_, ldx, Ri_[slot], ld_, d_, out, ldout, nullptr, info_, st_, true);
  }
  // One CholeskyQR pass: out = X R^{-1}, and a second pass when the first
  // Cholesky had to shift (gated on a device flag, so the launch sequence
  // stays static). A shifted factor still spans R(X) but leaves out far from
  // orthonormal, and the next pass over A would carry that conditioning into
  // its small directions. X is dead afterwards (it holds the second pass's
  // product). have_r0: the R factor is already in slot 0 (the probe) and the
  // probe's shift flag in gates[kInterGate].
  cudaError_t orth_inter(float* X, int64_t ldx, int64_t rows, float* out, int64_t ldout, bool have_r0 = false) {
    int* g = &gates[kInterGate];
    if (have_r0) {
      CK(apply_r0(X, ldx, rows, out, ldout));
    } else {
      CK(cudaMemsetAsync(g, 0, sizeof(int), st_));
      if (tc_on_ && rows > (int64_t)d_) {
        CK(tc_cqr(X, ldx, rows, out, ldout, 0, g, false));
      } else {
        CK(gram(X, ldx, rows, nullptr));
        CK(chol(0, g, nullptr, false));
        CK(trmm(X, ldx, rows, Ri_[0], out, ldout, nullptr));
      }
    }
    CK(gram(out, ldout, rows, g));
    CK(chol(1, nullptr, g, false));
    CK(gemm_f32_ex(false, rows, d_, d_, out, ldout, Ri_[1], ld_, X, ldx, 1, nullptr, nullptr, g, kGateSkip, true,
                   st_));
    return copy_matrix(rows, d_, X, ldx, out, ldout, st_, g);
  }
  // CholeskyQR2 plus a third pass gated on a shifted Cholesky (shifted
  // CholeskyQR3). X (rows x d) is overwritten; tmp holds rows x d (ld_);
  // Racc (optional, d x d, ld_) receives R = R3 R2 R1.
  cudaError_t orth_final(float* X, int64_t ldx, int64_t rows, float* out, int64_t ldout, float* tmp,
                         float* Racc, int slot, bool have_r0 = false) {
    int* g = &gates[slot];
    const bool want_r = Racc != nullptr;
    if (have_r0) {   // first pass from the probe's R (slot 0, gate in gates[0])
      CK(apply_r0(X, ldx, rows, tmp, ld_));
    } else if (tc_on_ && rows > (int64_t)d_) {
      // First pass on the tensor cores (BF16x3 Gram, exact-mode X R^{-1});
      // the second pass, which sets the orthogonality, stays in FP32.
      CK(tc_cqr(X, ldx, rows, tmp, ld_, 0, g, want_r));
    } else {
      CK(gram(X, ldx, rows, nullptr));
      CK(chol(0, g, nullptr, want_r));
      CK(trmm(X, ldx, rows, Ri_[0], tmp, ld_, nullptr));
    }
    CK(gram(tmp, ld_, rows, nullptr));
    CK(chol(1, g, nullptr, want_r));
    CK(trmm(tmp, ld_, rows, Ri_[1], X, ldx, nullptr));
    CK(gram(X, ldx, rows, g));
    CK(chol(2, nullptr, g, want_r));
    CK(trmm(X, ldx, rows, Ri_[2], out, ldout, g));
    if (Racc != nullptr) {
      // d x d products, split along K (their partials fit the Gram's buffer)
      const int sk = gemm_f32_splits(d_, d_, d_);
      CK(gemm_f32_ex(false, d_, d_, d_, R_[1], ld_, R_[0], ld_, Ra_, ld_, sk, part_, nullptr, nullptr,
                     kGateNone, true, st_));
      CK(gemm_f32_ex(false, d_, d_, d_, R_[2], ld_, Ra_, ld_, Racc, ld_, sk, part_, nullptr, nullptr,
                     kGateNone, true, st_));
    }
    return cudaSuccess;
  }

  double* scal = nullptr;
  int* gates = nullptr;

 private:
  int d_, dcap_;
  int64_t ld_;
  rqlp_opts o_;
  cudaStream_t st_ = nullptr;
  int* info_ = nullptr;
  float *G_ = nullptr, *R_[3] = {}, *Ri_[3] = {}, *Ra_ = nullptr, *part_ = nullptr;
  void* cstore_ = nullptr;
  TcEngine tc_, tcs_;
  bool tc_on_ = false;
  bool three_ = false;
  const SparseA* sp_ = nullptr;
  const SparseA* spt_ = nullptr;
};

struct Dims {
  int64_t m, n, lda, ldo;
  int k, p, q, d;
  bool learned = false;   // d = k + 20 is a capacity; the run picks p in {5, 10, 20}
};

struct Out {
  float* Q; int64_t ldq;
  float* L; int64_t ldl;
  float* P; int64_t ldp;
};

// Copy streams and events of the host-ingest entry points: created on first
// use per device and kept for the life of the process (host-side objects; no
// device memory).
constexpr int kIngestBlocks = 16;
struct IngestStreams {
  std::mutex busy;   // one host-ingest call per device at a time
  cudaStream_t copy[2];
  cudaEvent_t start;
  cudaEvent_t landed[kIngestBlocks];
};
IngestStreams* ingest_streams() {
  static std::mutex mu;
  static IngestStreams* per_dev[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (per_dev[dev] == nullptr) {
    IngestStreams* io = new IngestStreams();
    bool ok = cudaStreamCreateWithFlags(&io->copy[0], cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&io->copy[1], cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&io->start, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < kIngestBlocks; ++i)
      ok = cudaEventCreateWithFlags(&io->landed[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return nullptr;   // (the handles created so far are left to the process)
    per_dev[dev] = io;
  }
  return per_dev[dev];
}

// Parts per operand of the BF16X3 passes over A: the caller's choice, or
// automatically three when the oversampling p is below 5 or m n <= 2^27.
// Every pass rounds at ~2^-16 |A| |X| with two parts; what that does to
// |L_ii| grows with sigma_1 / sigma_i, with the inverse of the test matrix's
// leading block U_k^T Omega (the t = ||Omega~_2 Omega~_1^{-1}|| of Theorems
// 1-2, section 4.1; large when that block is nearly square, p < 5), and
// shrinks like K^(-1/2) as each entry sums more independently rounded terms.
// Measured against the FP64 oracle, two parts missed the 1e-4 |L_ii| bound on
// small problems (2.2e-4 at 705 x 1798, k = 41, p = 5) and at p = 0, and met
// it at 16384^2 and 20000^2 with p >= 5; three parts met it on all of them.
// p < 0: the oversampling is not known (one pass on its own, two parts
// unless the size says otherwise).
bool three_part_passes(const rqlp_opts& o, int64_t m, int64_t n, int p) {
  if (o.precision != RQLP_PREC_BF16X3) return false;
  if (o.bf16_parts != 0) return o.bf16_parts == 3;
  return (p >= 0 && p < 5) || m * n <= (int64_t(1) << 27);
}

// The whole chain for one matrix. Dims.d is the widest sketch the workspace
// serves; the learned form runs the chain at a narrower width.
class Plan {
 public:
  Plan(const Dims& dm, const rqlp_opts& o) : d_(dm), ops_(dm.d, o), o_(o) {
    ops_.set_three_part(three_part_passes(o, dm.m, dm.n, dm.learned ? 20 : dm.p));
  }

  size_t layout(Arena& ar) {
    const int64_t ld = ops_.ld(), dd = (int64_t)d_.d * ld, tall = std::max(d_.m, d_.n);
    Y_ = ar.take<float>(d_.n * ld);
    Z_ = ar.take<float>(d_.m * ld);
    Pt_ = ar.take<float>(d_.n * ld);
    T1_ = ar.take<float>(tall * ld);
    Rb_ = ar.take<float>(dd);
    Rh_ = ar.take<float>(dd);
    Ts_ = ar.take<float>(dd);
    Ts2_ = ar.take<float>(dd);
    Ph_ = ar.take<float>(dd);
    feat_ = ar.take<float>(RQLP_MLP_FEATURES);
    logits_ = ar.take<float>(RQLP_MLP_OUTPUTS);
    qp_ = ar.take<int>(2);
    // Split-K partial buffers for every width this plan may run at.
    size_t part = 0;
    const int lo = d_.learned ? std::max(1, d_.d - 15) : d_.d;
    for (int d = lo; d <= d_.d; ++d)
      part = std::max({part, Ops::pass_part_floats(d_.m, d_.n, d), Ops::orth_part_floats(d_.m, d),
                       Ops::orth_part_floats(d_.n, d), Ops::orth_part_floats(d, d)});
    if (o_.fused_power != 0 && o_.precision == RQLP_PREC_FP32)
      for (int d = lo; d <= d_.d; ++d) part = std::max(part, Ops::fused_part_floats(d_.m, d_.n, d));
    ops_.layout(ar, part, o_.precision == RQLP_PREC_BF16X3, d_.m, d_.n);
    return ar.off;
  }

  cudaError_t run(const float* A, const float* Om, const Out& out, int* info, double* diag, cudaStream_t st) {
    ops_.bind(st, info);
    CK(ops_.init());
    {
      Range r("rqlp: sketch Y = A^T Omega");
      // Sketch Y = A^T Omega (Algorithm 1 step 3); ||A||_F^2 rides along.
      CK(ops_.pass(true, A, d_.m, d_.n, d_.lda, Om, d_.ldo, Y_, ops_.ld(), &ops_.scal[0]));
    }
    return chain(A, d_.q, out, info, diag, st);
  }

  // The chain for a sparse A: its transpose (CSR) is built into csc_ws
  // first, then every pass is a sparse product.
  cudaError_t run_sparse(const SparseA& a, void* csc_ws, const float* Om, const Out& out, int* info, double* diag,
                         cudaStream_t st) {
    ops_.bind(st, info);
    CK(ops_.init());
    {
      Range r("rqlp: sparse transpose");
      CK(sparse_build_csc(a, csc_ws, &at_, info, st));
    }
    a_ = a;
    ops_.set_sparse(&a_, &at_);
    {
      Range r("rqlp: sketch Y = A^T Omega (sparse)");
      CK(ops_.pass(true, nullptr, d_.m, d_.n, d_.n, Om, d_.ldo, Y_, ops_.ld(), &ops_.scal[0]));
    }
    return chain(nullptr, d_.q, out, info, diag, st);
  }

  // Probe sketch of the full width, its R factor, features, the network's
  // error estimates and (q, p), all on the device. params == nullptr stops
  // after the features.
  cudaError_t probe(const float* A, const float* Om, double target, const float* params, int* info,
                    cudaStream_t st) {
    Range r("rqlp: probe sketch, features, (q, p)");
    ops_.bind(st, info);
    CK(ops_.init());
    ops_.set_d(d_.d);
    CK(ops_.pass(true, A, d_.m, d_.n, d_.lda, Om, d_.ldo, Y_, ops_.ld(), &ops_.scal[0]));
    CK(ops_.gram_chol(Y_, ops_.ld(), d_.n));
    CK(probe_features(ops_.R(0), ops_.ld(), d_.d, d_.k, std::min(d_.m, d_.n), feat_, st));
    if (params == nullptr) return cudaSuccess;
    CK(mlp_forward(params, feat_, 1, logits_, st));
    return predict_qp(logits_, params, info, target, d_.k, qp_, st);
  }
  const float* features() const { return feat_; }
  const int* qp() const { return qp_; }

  // The probe with A and Omega arriving from host memory: row blocks are
  // copied on the library's copy streams and each block's share of the
  // sketch, A_b^T Omega_b, runs as soon as it has landed (the sum over blocks
  // in FP32, in block order), so the copy of A overlaps its first pass.
  // dA (m x n, ld n) and dOm (m x ldo) receive the copies.
  cudaError_t probe_from_host(float* dA, float* dOm, int64_t ldo, const float* hA, int64_t hlda, const float* hOm,
                              int64_t hldo, double target, const float* params, int* info, cudaStream_t st) {
    Range r("rqlp: host ingest, probe sketch, features, (q, p)");
    ops_.bind(st, info);
    CK(ops_.init());
    ops_.set_d(d_.d);
    const int64_t m = d_.m, n = d_.n, ld = ops_.ld();
    IngestStreams* io = ingest_streams();
    if (io == nullptr) return cudaErrorInitializationError;
    const int nb = (int)std::min<int64_t>(kIngestBlocks, std::max<int64_t>(1, cdiv(m, 2048)));
    const int64_t brows = round_up(cdiv(m, nb), 64);
    const size_t F = sizeof(float);
    // the copy streams start after the work already on `st`
    CK(cudaEventRecord(io->start, st));
    for (int c = 0; c < 2; ++c) CK(cudaStreamWaitEvent(io->copy[c], io->start, 0));
    int b = 0;
    for (int64_t r0 = 0; r0 < m; r0 += brows, ++b) {
      const int64_t rows = std::min(brows, m - r0);
      cudaStream_t cs = io->copy[b & 1];
      CK(cudaMemcpy2DAsync(dA + r0 * n, n * F, hA + r0 * hlda, hlda * F, n * F, rows, cudaMemcpyHostToDevice, cs));
      CK(cudaMemcpy2DAsync(dOm + r0 * ldo, ldo * F, hOm + r0 * hldo, hldo * F, d_.d * F, rows,
                           cudaMemcpyHostToDevice, cs));
      CK(cudaEventRecord(io->landed[b], cs));
      CK(cudaStreamWaitEvent(st, io->landed[b], 0));
      float* dst = r0 == 0 ? Y_ : T1_;
      CK(ops_.pass_rows(dA, m, n, n, r0, rows, dOm + r0 * ldo, ldo, dst, ld));
      if (r0 > 0) CK(add_matrix(n, d_.d, T1_, ld, Y_, ld, st));
    }
    CK(ops_.gram_chol(Y_, ld, n));
    CK(probe_features(ops_.R(0), ld, d_.d, d_.k, std::min(m, n), feat_, st));
    CK(mlp_forward(params, feat_, 1, logits_, st));
    return predict_qp(logits_, params, info, target, d_.k, qp_, st);
  }

  // Continue from the probe with the predicted (q, p): the probe's first
  // k + p columns are the sketch A^T Omega_{k+p}.
  // Its R factor (slot 0) serves the chain's first orthonormalisation; the
  // probe's shift gate only matters when that one is the final CholeskyQR2.
  cudaError_t finish_learned(const float* A, int q, int p, const Out& out, int* info, double* diag,
                             cudaStream_t st) {
    ops_.set_d(d_.k + p);
    if (q > 0) {   // the probe's shift flag gates the second intermediate pass; gates[0] the final one
      CK(cudaMemcpyAsync(&ops_.gates[kInterGate], &ops_.gates[0], sizeof(int), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemsetAsync(&ops_.gates[0], 0, sizeof(int), st));
    }
    return chain(A, q, out, info, diag, st, true);
  }

 private:
  // From Y = A^T Omega (width ops_.d()) to Q, L, P.
  // have_r0: the R factor of Y is already in slot 0.
  cudaError_t chain(const float* A, int q, const Out& out, int* info, double* diag, cudaStream_t st,
                    bool have_r0 = false) {
    const int64_t m = d_.m, n = d_.n, lda = d_.lda, ld = ops_.ld();
    const int d = ops_.d();
    {
      Range r("rqlp: qf(Y)");
      if (q == 0) CK(ops_.orth_final(Y_, ld, n, Pt_, ld, T1_, nullptr, 0, have_r0));
      else CK(ops_.orth_inter(Y_, ld, n, Pt_, ld, have_r0));
    }
    for (int i = 1; i <= q; ++i) {
      Range r("rqlp: power pass");
      if (o_.fused_power != 0) {
        CK(ops_.power_fused(A, m, n, lda, Pt_, ld, Y_, ld, Z_, T1_));   // Y = A^T (A P~)
      } else {
        CK(ops_.pass(false, A, m, n, lda, Pt_, ld, Z_, ld, nullptr));   // Z = A P~
        CK(ops_.orth_inter(Z_, ld, m, T1_, ld));                        // Z = qf(Z), one pass
        CK(ops_.pass(true, A, m, n, lda, T1_, ld, Y_, ld, nullptr));    // Y = A^T Z
      }
      if (i == q) CK(ops_.orth_final(Y_, ld, n, Pt_, ld, T1_, nullptr, 0));
      else CK(ops_.orth_inter(Y_, ld, n, Pt_, ld));
    }
    if (o_.literal_step5 != 0) {
      // Algorithm 1 steps 4-5 as printed: Q = qf(A P~), then the QR of
      // (Q^T A)^T = A^T Q (a third pass over A) gives P and R', L = R'^T.
      // Q L P^T = Q Q^T A, so ||A - Q L P^T||^2 = ||A||^2 - ||L||^2 as well.
      Range r("rqlp: qf(A P~), qr(A^T Q), L");
      CK(ops_.pass(false, A, m, n, lda, Pt_, ld, Z_, ld, nullptr));
      CK(ops_.orth_final(Z_, ld, m, out.Q, out.ldq, T1_, nullptr, 1));
      CK(ops_.pass(true, A, m, n, lda, out.Q, out.ldq, Y_, ld, nullptr));
      CK(ops_.orth_final(Y_, ld, n, out.P, out.ldp, T1_, Rh_, 2));
      CK(write_L(d, Rh_, ld, out.L, out.ldl, &ops_.scal[1], st));
      return finish_diag(ops_.scal, diag, info, st);
    }
    // (Q, R) = qr(A P~)  (Algorithm 1 step 4)
    Range r("rqlp: qr(A P~), qr(R^T), L, P");
    CK(ops_.pass(false, A, m, n, lda, Pt_, ld, Z_, ld, nullptr));
    CK(ops_.orth_final(Z_, ld, m, out.Q, out.ldq, T1_, Rb_, 1));
    // (P^, R^) = qr(R^T), L = R^^T  (step 5 applied to the d x d factor)
    CK(transpose_small(d, Rb_, ld, Ts_, ld, st));
    CK(ops_.orth_final(Ts_, ld, d, Ph_, ld, Ts2_, Rh_, 2));
    CK(write_L(d, Rh_, ld, out.L, out.ldl, &ops_.scal[1], st));
    // P = P~ P^ (FP32: P's entries are ~sqrt(d) times smaller than |P~| |P^|,
    // more than the tensor cores' accumulation leaves room for)
    CK(gemm_f32_ex(false, n, d, d, Pt_, ld, Ph_, ld, out.P, out.ldp, 1, nullptr, nullptr, nullptr, kGateNone,
                   false, st));
    return finish_diag(ops_.scal, diag, info, st);
  }

  Dims d_;
  Ops ops_;
  rqlp_opts o_;
  SparseA a_{}, at_{};
  float *Y_ = nullptr, *Z_ = nullptr, *Pt_ = nullptr, *T1_ = nullptr;
  float *Rb_ = nullptr, *Rh_ = nullptr, *Ts_ = nullptr, *Ts2_ = nullptr, *Ph_ = nullptr;
  float *feat_ = nullptr, *logits_ = nullptr;
  int* qp_ = nullptr;
};

rqlp_opts resolve(const rqlp_opts* o) {
  rqlp_opts r;
  rqlp_default_opts(&r);
  if (o != nullptr) r = *o;
  return r;
}

bool valid_opts(const rqlp_opts& o) {
  if (o.precision != RQLP_PREC_FP32 && o.precision != RQLP_PREC_BF16X3) return false;
  if (o.small_fp64 != 0 && o.small_fp64 != 1) return false;
  if (o.test_stall != 0) return false;   // the hook is the batched form's only
  if (o.bf16_parts != 0 && (o.precision != RQLP_PREC_BF16X3 || (o.bf16_parts != 2 && o.bf16_parts != 3)))
    return false;
  if (o.literal_step5 != 0 && o.literal_step5 != 1) return false;
  if (o.fused_power != 0 && o.fused_power != 1) return false;
  for (int i = 0; i < 2; ++i)
    if (o.reserved[i] != 0) return false;
  return true;
}

bool valid_sizes(int64_t m, int64_t n, int k, int p, int q) {
  if (m <= 0 || n <= 0 || k < 1 || p < 0 || q < 0 || q > 64) return false;
  const int64_t d = (int64_t)k + p;
  return d <= std::min(m, n) && d <= RQLP_MAX_D;
}

Dims make_dims(int64_t m, int64_t n, int64_t lda, int k, int p, int q, int64_t ldo) {
  Dims dm;
  dm.m = m; dm.n = n; dm.lda = lda; dm.ldo = ldo;
  dm.k = k; dm.p = p; dm.q = q; dm.d = k + p;
  return dm;
}

size_t plan_bytes(const Dims& dm, const rqlp_opts& o) {
  Arena ar;
  ar.dry = true;
  Plan pl(dm, o);
  return pl.layout(ar);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

Arena arena_over(void* ws, size_t bytes) {
  Arena ar;
  ar.base = static_cast<char*>(ws);
  ar.cap = bytes;
  return ar;
}

size_t sketch_bytes(int64_t m, int64_t n, int d, const rqlp_opts& o) {
  Arena ar;
  ar.dry = true;
  Ops ops(d, o);
  ops.set_three_part(three_part_passes(o, m, n, -1));
  ops.layout(ar, Ops::pass_part_floats(m, n, d), o.precision == RQLP_PREC_BF16X3, m, n);
  return ar.off;
}

size_t orth_bytes(int64_t rows, int d, const rqlp_opts& o) {
  Arena ar;
  ar.dry = true;
  const int64_t ld = round_up(d, 4);
  ar.take<float>(rows * ld);
  ar.take<float>((int64_t)d * ld);
  Ops ops(d, o);
  ops.layout(ar, Ops::orth_part_floats(rows, d), false, rows, d);
  return ar.off;
}

}  // namespace
}  // namespace rqlp

using namespace rqlp;

extern "C" {

void rqlp_default_opts(rqlp_opts* opts) {
  if (opts == nullptr) return;
  std::memset(opts, 0, sizeof(*opts));
  opts->precision = RQLP_PREC_FP32;
  opts->small_fp64 = 0;
}

size_t rqlp_workspace_bytes(int64_t m, int64_t n, int k, int p, int q, const rqlp_opts* opts) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_sizes(m, n, k, p, q)) return 0;
  return plan_bytes(make_dims(m, n, n, k, p, q, k + p), o);
}

rqlp_status rqlp_factor(const float* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                        const float* Omega, int64_t ldo, float* Q, int64_t ldq, float* L, int64_t ldl,
                        float* P, int64_t ldp, void* workspace, size_t ws_bytes, int* d_info, double* d_diag,
                        const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_sizes(m, n, k, p, q)) return RQLP_ERR_ARG;
  const int d = k + p;
  if (A == nullptr || Omega == nullptr || Q == nullptr || L == nullptr || P == nullptr || d_info == nullptr)
    return RQLP_ERR_ARG;
  if (lda < n || ldo < d || ldq < d || ldl < d || ldp < d) return RQLP_ERR_ARG;
  if (o.precision == RQLP_PREC_BF16X3 && !tc_supported(A, lda, Omega, ldo)) return RQLP_ERR_UNSUPPORTED;
  Dims dm = make_dims(m, n, lda, k, p, q, ldo);
  const size_t need = plan_bytes(dm, o);
  if (workspace == nullptr || ws_bytes < need || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  Arena ar = arena_over(workspace, ws_bytes);
  Plan pl(dm, o);
  pl.layout(ar);
  Out out{Q, ldq, L, ldl, P, ldp};
  cudaError_t e = pl.run(A, Omega, out, d_info, d_diag, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_host_workspace_bytes(int64_t m, int64_t n, int k, int p, int q, const rqlp_opts* opts) {
  size_t core = rqlp_workspace_bytes(m, n, k, p, q, opts);
  if (core == 0) return 0;
  const int64_t d = k + p, ld = round_up(d, 4);
  Arena ar;
  ar.dry = true;
  ar.take<float>((size_t)(m * n));
  ar.take<float>((size_t)(m * ld));
  ar.take<float>((size_t)(m * ld));
  ar.take<float>((size_t)(d * ld));
  ar.take<float>((size_t)(n * ld));
  ar.take<int>(RQLP_INFO_INTS);
  ar.take<double>(RQLP_DIAG_DOUBLES);
  return round_up((int64_t)ar.off, 256) + core;
}

rqlp_status rqlp_factor_host(const float* hA, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                             const float* hOmega, int64_t ldo, float* hQ, int64_t ldq, float* hL, int64_t ldl,
                             float* hP, int64_t ldp, void* workspace, size_t ws_bytes, int* h_info,
                             double* h_diag, const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_sizes(m, n, k, p, q)) return RQLP_ERR_ARG;
  const int64_t d = k + p, ld = round_up(d, 4);
  if (hA == nullptr || hOmega == nullptr || hQ == nullptr || hL == nullptr || hP == nullptr ||
      h_info == nullptr)
    return RQLP_ERR_ARG;
  if (lda < n || ldo < d || ldq < d || ldl < d || ldp < d) return RQLP_ERR_ARG;
  const size_t need = rqlp_host_workspace_bytes(m, n, k, p, q, &o);
  if (workspace == nullptr || ws_bytes < need || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena ar = arena_over(workspace, ws_bytes);
  float* A = ar.take<float>((size_t)(m * n));
  float* Om = ar.take<float>((size_t)(m * ld));
  float* Q = ar.take<float>((size_t)(m * ld));
  float* L = ar.take<float>((size_t)(d * ld));
  float* P = ar.take<float>((size_t)(n * ld));
  int* info = ar.take<int>(RQLP_INFO_INTS);
  double* diag = ar.take<double>(RQLP_DIAG_DOUBLES);
  const size_t off = (size_t)round_up((int64_t)ar.off, 256);
  void* core = static_cast<char*>(workspace) + off;
  const size_t F = sizeof(float);
  // Once a copy from the caller's host buffers is enqueued, every return
  // waits for the stream first, so no copy is still reading or writing them
  // when the caller gets control back (error paths included).
  auto fail = [st](rqlp_status s) {
    (void)cudaStreamSynchronize(st);
    return s;
  };
  if (cudaMemcpy2DAsync(A, n * F, hA, lda * F, n * F, m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpy2DAsync(Om, ld * F, hOmega, ldo * F, d * F, m, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(RQLP_ERR_CUDA);
  rqlp_status s = rqlp_factor(A, m, n, n, k, p, q, Om, ld, Q, ld, L, ld, P, ld, core, ws_bytes - off, info,
                              diag, &o, stream);
  if (s != RQLP_OK) return fail(s);
  if (cudaMemcpy2DAsync(hQ, ldq * F, Q, ld * F, d * F, m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(hL, ldl * F, L, ld * F, d * F, d, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(hP, ldp * F, P, ld * F, d * F, n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(h_info, info, RQLP_INFO_INTS * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(RQLP_ERR_CUDA);
  if (h_diag != nullptr &&
      cudaMemcpyAsync(h_diag, diag, RQLP_DIAG_DOUBLES * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
    return fail(RQLP_ERR_CUDA);
  return cudaStreamSynchronize(st) == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_sketch_workspace_bytes(int trans, int64_t m, int64_t n, int d, const rqlp_opts* opts) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || (trans != 0 && trans != 1) || m <= 0 || n <= 0 || d < 1 || d > RQLP_MAX_D) return 0;
  return sketch_bytes(m, n, d, o);
}

rqlp_status rqlp_sketch(int trans, const float* A, int64_t m, int64_t n, int64_t lda, const float* X,
                        int64_t ldx, int d, float* Y, int64_t ldy, void* workspace, size_t ws_bytes,
                        const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  const size_t need = rqlp_sketch_workspace_bytes(trans, m, n, d, &o);
  if (need == 0 || A == nullptr || X == nullptr || Y == nullptr || lda < n || ldx < d || ldy < d)
    return RQLP_ERR_ARG;
  if (o.precision == RQLP_PREC_BF16X3 && !tc_supported(A, lda, X, ldx)) return RQLP_ERR_UNSUPPORTED;
  if (workspace == nullptr || ws_bytes < need || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  Arena ar = arena_over(workspace, ws_bytes);
  Ops ops(d, o);
  ops.set_three_part(three_part_passes(o, m, n, -1));
  ops.layout(ar, Ops::pass_part_floats(m, n, d), o.precision == RQLP_PREC_BF16X3, m, n);
  ops.bind(static_cast<cudaStream_t>(stream), nullptr);
  cudaError_t e = ops.pass(trans == 1, A, m, n, lda, X, ldx, Y, ldy, nullptr);
  return e == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_orth_workspace_bytes(int64_t rows, int d, const rqlp_opts* opts) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || d < 1 || d > RQLP_MAX_D || rows < d) return 0;
  return orth_bytes(rows, d, o);
}

rqlp_status rqlp_orth(float* X, int64_t rows, int d, int64_t ldx, float* R, int64_t ldr, void* workspace,
                      size_t ws_bytes, int* d_info, const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  const size_t need = rqlp_orth_workspace_bytes(rows, d, &o);
  if (need == 0 || X == nullptr || d_info == nullptr || ldx < d || (R != nullptr && ldr < d)) return RQLP_ERR_ARG;
  if (workspace == nullptr || ws_bytes < need || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  Arena ar = arena_over(workspace, ws_bytes);
  const int64_t ld = round_up(d, 4);
  float* tmp = ar.take<float>(rows * ld);
  float* Racc = ar.take<float>((int64_t)d * ld);
  Ops ops(d, o);
  ops.layout(ar, Ops::orth_part_floats(rows, d), false, rows, d);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ops.bind(st, d_info);
  // The last pass reads X, so it writes tmp (free again by then) and Q is
  // copied back into X afterwards.
  cudaError_t e = ops.init();
  if (e == cudaSuccess) e = ops.orth_final(X, ldx, rows, tmp, ld, tmp, Racc, 0);
  if (e == cudaSuccess) e = copy_matrix(rows, d, tmp, ld, X, ldx, st);
  if (e == cudaSuccess && R != nullptr) e = copy_matrix(d, d, Racc, ld, R, ldr, st);
  return e == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_mlp_workspace_bytes(int batch) {
  if (batch <= 0) return 0;
  return mlp_workspace_floats(batch) * sizeof(float);
}

rqlp_status rqlp_mlp_forward(const float* params, const float* X, int batch, float* logits, void* stream) {
  if (params == nullptr || X == nullptr || logits == nullptr || batch <= 0) return RQLP_ERR_ARG;
  return mlp_forward(params, X, batch, logits, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RQLP_OK
                                                                                                 : RQLP_ERR_CUDA;
}

rqlp_status rqlp_mlp_grad(const float* params, const float* X, const float* Y, int batch, float* grad, float* loss,
                          void* workspace, size_t ws_bytes, void* stream) {
  if (params == nullptr || X == nullptr || Y == nullptr || grad == nullptr || batch <= 0) return RQLP_ERR_ARG;
  if (workspace == nullptr || ws_bytes < rqlp_mlp_workspace_bytes(batch) || !aligned(workspace, 16))
    return RQLP_ERR_WORKSPACE;
  return mlp_grad(params, X, Y, batch, grad, loss, workspace, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? RQLP_OK
             : RQLP_ERR_CUDA;
}

rqlp_status rqlp_mlp_adam(float* params, const float* grad, float* m1, float* m2, int n, float lr, float beta1,
                          float beta2, float eps, int step, void* stream) {
  if (params == nullptr || grad == nullptr || m1 == nullptr || m2 == nullptr || n <= 0 || step < 1)
    return RQLP_ERR_ARG;
  return mlp_adam(params, grad, m1, m2, n, lr, beta1, beta2, eps, step, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? RQLP_OK
             : RQLP_ERR_CUDA;
}

namespace {
bool valid_learned(int64_t m, int64_t n, int k) { return valid_sizes(m, n, k, 20, 0); }
bool valid_target(double t) { return t > 0.0 && t < 1.0; }
Dims learned_dims(int64_t m, int64_t n, int64_t lda, int k, int64_t ldo) {
  Dims dm = make_dims(m, n, lda, k, 20, 4, ldo);
  dm.learned = true;
  return dm;
}
}  // namespace

size_t rqlp_learned_workspace_bytes(int64_t m, int64_t n, int k, const rqlp_opts* opts) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_learned(m, n, k)) return 0;
  return plan_bytes(learned_dims(m, n, n, k, k + 20), o);
}

static rqlp_status probe_common(const float* A, int64_t m, int64_t n, int64_t lda, int k, const float* Omega,
                                int64_t ldo, double target, const float* params, float* feat, int* d_qp,
                                void* workspace, size_t ws_bytes, int* d_info, const rqlp_opts* opts,
                                void* stream) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_learned(m, n, k) || !valid_target(target) || A == nullptr || Omega == nullptr ||
      d_info == nullptr)
    return RQLP_ERR_ARG;
  if (lda < n || ldo < k + 20) return RQLP_ERR_ARG;
  if (o.precision == RQLP_PREC_BF16X3 && !tc_supported(A, lda, Omega, ldo)) return RQLP_ERR_UNSUPPORTED;
  Dims dm = learned_dims(m, n, lda, k, ldo);
  if (workspace == nullptr || ws_bytes < plan_bytes(dm, o) || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  Arena ar = arena_over(workspace, ws_bytes);
  Plan pl(dm, o);
  pl.layout(ar);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl.probe(A, Omega, target, params, d_info, st) != cudaSuccess) return RQLP_ERR_CUDA;
  if (feat != nullptr &&
      copy_matrix(1, RQLP_MLP_FEATURES, pl.features(), RQLP_MLP_FEATURES, feat, RQLP_MLP_FEATURES, st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  if (d_qp != nullptr && cudaMemcpyAsync(d_qp, pl.qp(), 2 * sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  return RQLP_OK;
}

rqlp_status rqlp_probe_features(const float* A, int64_t m, int64_t n, int64_t lda, int k, const float* Omega,
                                int64_t ldo, float* feat, void* workspace, size_t ws_bytes, int* d_info,
                                const rqlp_opts* opts, void* stream) {
  if (feat == nullptr) return RQLP_ERR_ARG;
  // no request is involved in the features; any valid one passes the check
  return probe_common(A, m, n, lda, k, Omega, ldo, 0.5, nullptr, feat, nullptr, workspace, ws_bytes, d_info,
                      opts, stream);
}

rqlp_status rqlp_predict_qp(const float* A, int64_t m, int64_t n, int64_t lda, int k, const float* Omega,
                            int64_t ldo, double target, const float* params, int* d_qp, void* workspace,
                            size_t ws_bytes, int* d_info, const rqlp_opts* opts, void* stream) {
  if (params == nullptr || d_qp == nullptr) return RQLP_ERR_ARG;
  return probe_common(A, m, n, lda, k, Omega, ldo, target, params, nullptr, d_qp, workspace, ws_bytes, d_info,
                      opts, stream);
}

rqlp_status rqlp_factor_learned(const float* A, int64_t m, int64_t n, int64_t lda, int k, const float* Omega,
                                int64_t ldo, double target, const float* params, float* Q, int64_t ldq, float* L,
                                int64_t ldl, float* P, int64_t ldp, void* workspace, size_t ws_bytes, int* d_info,
                                double* d_diag, int* h_qp, const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_learned(m, n, k) || !valid_target(target) || A == nullptr || Omega == nullptr ||
      params == nullptr || Q == nullptr || L == nullptr || P == nullptr || d_info == nullptr || h_qp == nullptr)
    return RQLP_ERR_ARG;
  const int dmax = k + 20;
  if (lda < n || ldo < dmax || ldq < dmax || ldl < dmax || ldp < dmax) return RQLP_ERR_ARG;
  if (o.precision == RQLP_PREC_BF16X3 && !tc_supported(A, lda, Omega, ldo)) return RQLP_ERR_UNSUPPORTED;
  Dims dm = learned_dims(m, n, lda, k, ldo);
  if (workspace == nullptr || ws_bytes < plan_bytes(dm, o) || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  Arena ar = arena_over(workspace, ws_bytes);
  Plan pl(dm, o);
  pl.layout(ar);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl.probe(A, Omega, target, params, d_info, st) != cudaSuccess) return RQLP_ERR_CUDA;
  int qp[2] = {-1, -1};
  if (cudaMemcpyAsync(qp, pl.qp(), sizeof(qp), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  if (qp[0] < 0 || qp[0] > 4 || (qp[1] != 5 && qp[1] != 10 && qp[1] != 20)) return RQLP_ERR_CUDA;
  h_qp[0] = qp[0];
  h_qp[1] = qp[1];
  Out out{Q, ldq, L, ldl, P, ldp};
  return pl.finish_learned(A, qp[0], qp[1], out, d_info, d_diag, st) == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

size_t rqlp_learned_host_workspace_bytes(int64_t m, int64_t n, int k, const rqlp_opts* opts) {
  const size_t core = rqlp_learned_workspace_bytes(m, n, k, opts);
  if (core == 0) return 0;
  const int64_t w = k + 20, ld = round_up(w, 4);
  Arena ar;
  ar.dry = true;
  ar.take<float>((size_t)(m * n));       // A
  ar.take<float>((size_t)(m * ld));      // Omega
  ar.take<float>((size_t)(m * ld));      // Q
  ar.take<float>((size_t)(w * ld));      // L
  ar.take<float>((size_t)(n * ld));      // P
  ar.take<int>(RQLP_INFO_INTS);
  ar.take<double>(RQLP_DIAG_DOUBLES);
  return round_up((int64_t)ar.off, 256) + core;
}

rqlp_status rqlp_factor_learned_host(const float* hA, int64_t m, int64_t n, int64_t lda, int k, const float* hOmega,
                                     int64_t ldo, double target, const float* params, float* hQ, int64_t ldq,
                                     float* hL, int64_t ldl, float* hP, int64_t ldp, void* workspace,
                                     size_t ws_bytes, int* h_info, double* h_diag, int* h_qp,
                                     const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  if (!valid_opts(o) || !valid_learned(m, n, k) || !valid_target(target) || hA == nullptr || hOmega == nullptr ||
      params == nullptr || hQ == nullptr || hL == nullptr || hP == nullptr || h_info == nullptr || h_qp == nullptr)
    return RQLP_ERR_ARG;
  const int64_t w = k + 20, ld = round_up(w, 4);
  if (lda < n || ldo < w || ldq < w || ldl < w || ldp < w) return RQLP_ERR_ARG;
  if (o.precision == RQLP_PREC_BF16X3 && !tc_supported(nullptr, 0, nullptr, 0)) return RQLP_ERR_UNSUPPORTED;
  const size_t need = rqlp_learned_host_workspace_bytes(m, n, k, &o);
  if (workspace == nullptr || ws_bytes < need || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  IngestStreams* io = ingest_streams();
  if (io == nullptr) return RQLP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(io->busy);
  Arena ar = arena_over(workspace, ws_bytes);
  float* A = ar.take<float>((size_t)(m * n));
  float* Om = ar.take<float>((size_t)(m * ld));
  float* Q = ar.take<float>((size_t)(m * ld));
  float* L = ar.take<float>((size_t)(w * ld));
  float* P = ar.take<float>((size_t)(n * ld));
  int* info = ar.take<int>(RQLP_INFO_INTS);
  double* diag = ar.take<double>(RQLP_DIAG_DOUBLES);
  const size_t off = (size_t)round_up((int64_t)ar.off, 256);
  Arena core = arena_over(static_cast<char*>(workspace) + off, ws_bytes - off);
  Dims dm = learned_dims(m, n, n, k, ld);
  Plan pl(dm, o);
  pl.layout(core);
  // Once a copy from the caller's host buffers is enqueued, every return
  // waits for the device first (the copies run on the library's streams).
  auto fail = [](rqlp_status s) {
    (void)cudaDeviceSynchronize();
    return s;
  };
  if (pl.probe_from_host(A, Om, ld, hA, lda, hOmega, ldo, target, params, info, st) != cudaSuccess)
    return fail(RQLP_ERR_CUDA);
  int qp[2] = {-1, -1};
  if (cudaMemcpyAsync(qp, pl.qp(), sizeof(qp), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(RQLP_ERR_CUDA);
  if (qp[0] < 0 || qp[0] > 4 || (qp[1] != 5 && qp[1] != 10 && qp[1] != 20)) return fail(RQLP_ERR_CUDA);
  h_qp[0] = qp[0];
  h_qp[1] = qp[1];
  const int64_t d = k + qp[1];
  Out out{Q, ld, L, ld, P, ld};
  const size_t F = sizeof(float);
  if (pl.finish_learned(A, qp[0], qp[1], out, info, diag, st) != cudaSuccess ||
      cudaMemcpy2DAsync(hQ, ldq * F, Q, ld * F, d * F, m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(hL, ldl * F, L, ld * F, d * F, d, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(hP, ldp * F, P, ld * F, d * F, n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(h_info, info, RQLP_INFO_INTS * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (h_diag != nullptr &&
       cudaMemcpyAsync(h_diag, diag, RQLP_DIAG_DOUBLES * sizeof(double), cudaMemcpyDeviceToHost, st) !=
           cudaSuccess))
    return fail(RQLP_ERR_CUDA);
  return cudaStreamSynchronize(st) == cudaSuccess ? RQLP_OK : fail(RQLP_ERR_CUDA);
}

namespace {
bool valid_csr(const rqlp_csr* A) {
  return A != nullptr && A->m > 0 && A->n > 0 && A->nnz >= 0 && A->row_ptr != nullptr &&
         (A->nnz == 0 || (A->col_idx != nullptr && A->vals != nullptr)) && A->nnz < (int64_t(1) << 31);
}
}  // namespace

size_t rqlp_sparse_workspace_bytes(const rqlp_csr* A, int k, int p, int q, const rqlp_opts* opts) {
  rqlp_opts o = resolve(opts);
  if (!valid_csr(A) || !valid_opts(o) || o.precision != RQLP_PREC_FP32 || o.literal_step5 != 0 ||
      o.fused_power != 0 || !valid_sizes(A->m, A->n, k, p, q))
    return 0;
  return round_up((int64_t)plan_bytes(make_dims(A->m, A->n, A->n, k, p, q, k + p), o), 256) +
         sparse_csc_bytes(A->n, A->nnz);
}

rqlp_status rqlp_factor_sparse(const rqlp_csr* A, int k, int p, int q, const float* Omega, int64_t ldo, float* Q,
                               int64_t ldq, float* L, int64_t ldl, float* P, int64_t ldp, void* workspace,
                               size_t ws_bytes, int* d_info, double* d_diag, const rqlp_opts* opts, void* stream) {
  rqlp_opts o = resolve(opts);
  if (!valid_csr(A) || !valid_opts(o) || !valid_sizes(A->m, A->n, k, p, q)) return RQLP_ERR_ARG;
  if (o.precision != RQLP_PREC_FP32 || o.literal_step5 != 0 || o.fused_power != 0) return RQLP_ERR_UNSUPPORTED;
  const int d = k + p;
  if (Omega == nullptr || Q == nullptr || L == nullptr || P == nullptr || d_info == nullptr) return RQLP_ERR_ARG;
  if (ldo < d || ldq < d || ldl < d || ldp < d) return RQLP_ERR_ARG;
  const size_t need = rqlp_sparse_workspace_bytes(A, k, p, q, &o);
  if (workspace == nullptr || ws_bytes < need || !aligned(workspace, 256)) return RQLP_ERR_WORKSPACE;
  Dims dm = make_dims(A->m, A->n, A->n, k, p, q, ldo);
  const size_t core = (size_t)round_up((int64_t)plan_bytes(dm, o), 256);
  Arena ar = arena_over(workspace, core);
  Plan pl(dm, o);
  pl.layout(ar);
  SparseA a{A->m, A->n, A->nnz, A->row_ptr, A->col_idx, A->vals};
  Out out{Q, ldq, L, ldl, P, ldp};
  cudaError_t e = pl.run_sparse(a, static_cast<char*>(workspace) + core, Omega, out, d_info, d_diag,
                                static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

const char* rqlp_status_string(int status) {
  switch (status) {
    case RQLP_OK: return "ok";
    case RQLP_ERR_ARG: return "invalid argument";
    case RQLP_ERR_CUDA: return "CUDA error";
    case RQLP_ERR_BREAKDOWN: return "Cholesky breakdown (rank-deficient input)";
    case RQLP_ERR_NONFINITE: return "non-finite input";
    case RQLP_ERR_TIMEOUT: return "device wait timed out";
    case RQLP_ERR_WORKSPACE: return "workspace too small or misaligned";
    case RQLP_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int rqlp_version(void) { return 100; }

}  // extern "C"
