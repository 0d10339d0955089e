/*
 * rqlp.h -- C ABI of the GB300 (sm_103a) Rand-QLP library.
 *
 * Rand-QLP (Kaloorazi, Liu, Chen, de Lamare, arXiv 2110.01011) factors an
 * m x n matrix A as A ~= Q L P^T with Q and P orthonormal and L lower
 * triangular whose diagonal tracks the singular values of A (section 3.1,
 * Algorithm 1). This library computes the truncated chain with d = k + p
 * sketch columns and q power passes:
 *
 *   Y  = A^T Omega                         (Algorithm 1 step 3, Omega m x d)
 *   P~ = qf(Y)                             (orth via unpivoted QR, section 2)
 *   q times:  Z = qf(A P~),  P~ = qf(A^T Z)   (power passes)
 *   (Q, R)   = qr(A P~)                    (Algorithm 1 step 4)
 *   (P^, R^) = qr(R^T),  L = R^^T,  P = P~ P^   (step 5 on the d x d R)
 *
 * qf(.) is the Q factor of the thin QR with R's diagonal made positive, so
 * every factor is unique for full-rank inputs. With d = n and q = 0 the chain
 * is Algorithm 1 exactly.
 *
 * Conventions shared by every entry point:
 *  - Matrices are row-major FP32 with an explicit leading dimension (elements
 *    between consecutive rows, >= the column count).
 *  - Device pointers point to memory of the current CUDA device; the caller
 *    owns every buffer, including the workspace. The library allocates no
 *    device memory in rqlp_factor / rqlp_factor_batched.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = the
 *    legacy default stream) without host synchronisation, so calls can be
 *    captured into a CUDA graph. The return value reports argument and launch
 *    errors synchronously; numerical failures are written to the device
 *    array `d_info` (read it after synchronising the stream).
 *  - Sizes: 1 <= k, p >= 0, q >= 0, d = k + p <= min(m, n), d <= RQLP_MAX_D.
 *    Anything else returns RQLP_ERR_ARG and enqueues nothing.
 */
#ifndef RQLP_H
#define RQLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RQLP_MAX_D 256

typedef enum {
  RQLP_OK = 0,
  RQLP_ERR_ARG = 1,        /* invalid size, stride, pointer or option      */
  RQLP_ERR_CUDA = 2,       /* a CUDA launch or API call failed              */
  RQLP_ERR_BREAKDOWN = 3,  /* Cholesky breakdown even after the shift        */
  RQLP_ERR_NONFINITE = 4,  /* NaN/Inf met in A or Omega                      */
  RQLP_ERR_TIMEOUT = 5,    /* a bounded device wait gave up                  */
  RQLP_ERR_WORKSPACE = 6,  /* workspace too small or misaligned              */
  RQLP_ERR_UNSUPPORTED = 7 /* option not available on this device/build      */
} rqlp_status;

/* Arithmetic of the passes over A (the four dense products per power pass). */
typedef enum {
  RQLP_PREC_FP32 = 0,   /* FP32 FFMA on the CUDA cores                        */
  RQLP_PREC_BF16X3 = 1  /* tensor cores: A = A_hi + A_lo and X = X_hi + X_lo  */
                        /* in BF16, products hi*hi + hi*lo + lo*hi, FP32 acc. */
} rqlp_precision;

typedef struct {
  int precision;   /* rqlp_precision                                          */
  int small_fp64;  /* 1: d x d Cholesky factors in FP64 (slow on GB300);       */
                   /* 0: FP32 with an automatic diagonal shift on breakdown    */
  int test_stall;  /* fault-injection hook for tests, 0 in normal use: with    */
                   /* the BF16X3 batched form, 1 makes CTA 0 of the batch's   */
                   /* first grouped pass over A withhold its first stage's    */
                   /* loads, so that its bounded waits run out (~2 s each)    */
                   /* and the first problem's status row reports              */
                   /* RQLP_ERR_TIMEOUT; must be 0 for every other entry point */
  int bf16_parts;  /* BF16X3 only (0 with FP32): BF16 parts per operand of   */
                   /* the passes over A. 2: A = A_hi + A_lo, X = X_hi + X_lo, */
                   /* three products, error ~2^-16 |A| |X| per pass; 3: a    */
                   /* third part each (A_lo2 = bf16(A - A_hi - A_lo)), the   */
                   /* six products above 2^-24, FP32-level error at twice    */
                   /* the MMA work and 1.5x the bytes of the split A;        */
                   /* 0: automatic: three parts when p < 5 or m n <= 2^27,  */
                   /* else two (the batched form: three parts)               */
  int literal_step5; /* 0: step 5 on the d x d R, (P^, R^) = qr(R^T),         */
                   /* L = R^^T, P = P~ P^ (no third pass over A); 1: step 5 */
                   /* as Algorithm 1 prints it, (P, R') = qr((Q^T A)^T) =   */
                   /* qr(A^T Q), L = R'^T: a third pass over A. The two     */
                   /* agree when rank(A) <= d or d = n; with d = n, q = 0   */
                   /* and 1 the chain is Algorithm 1 as printed. Single-    */
                   /* matrix entry points only (0 for the batched form)     */
  int fused_power; /* 1: each power pass as Y = A^T (A P~) by row panels of A */
                   /* small enough to stay in L2, Z = A P~ not              */
                   /* orthonormalised (its span is all the next product     */
                   /* needs): one pass over A from HBM per power pass       */
                   /* instead of two. Measured slower than the two passes   */
                   /* at every shape tried (200000 x 500: 6.2 vs 5.8 ms;    */
                   /* 20000 x 20000: 12.8 vs 5.3 ms): an L2-sized panel     */
                   /* holds few 128-row tiles, and each panel writes a      */
                   /* full n x d partial of Y.                              */
                   /* 0: the two passes with qf(Z) between (default).       */
                   /* Dense single-matrix entry points only                 */
  int reserved[2]; /* must be zero                                            */
} rqlp_opts;

/* d_info layout written by rqlp_factor (2 ints): [0] = rqlp_status of the
 * numerical phase (RQLP_OK, RQLP_ERR_BREAKDOWN, RQLP_ERR_NONFINITE),
 * [1] = detail (1-based Cholesky column of the first breakdown, else 0). */
#define RQLP_INFO_INTS 2

/* d_diag layout (4 doubles, optional): [0] = ||A||_F^2, [1] = ||L||_F^2,
 * [2] = ||A - Q L P^T||_F^2 = [0] - [1] (Q L P^T = A P~ P~^T is the orthogonal
 * projection of A's rows on R(P~)), [3] = number of shifted Cholesky passes. */
#define RQLP_DIAG_DOUBLES 4

/* Opts with every field at its default (FP32 passes, FP32 small factors). */
void rqlp_default_opts(rqlp_opts* opts);

/* Bytes of device workspace rqlp_factor needs for these sizes and options
 * (0 when the arguments are invalid). Depends on the current device's SM
 * count; query it on the device that will run the factorisation. */
size_t rqlp_workspace_bytes(int64_t m, int64_t n, int k, int p, int q,
                            const rqlp_opts* opts);

/* Factor A (m x n, device, lda) with the Gaussian test matrix Omega
 * (m x d, device, ldo), d = k + p, q power passes. Writes
 *   Q (m x d, ldq): orthonormal columns;
 *   L (d x d, ldl): lower triangular with positive diagonal, strict upper
 *                   part written as 0;
 *   P (n x d, ldp): orthonormal columns,
 * such that Q L P^T = A P~ P~^T ~= A. In the BF16X3 form the low parts'
 * products accumulate in a TMEM accumulator apart from A_hi X_hi (added with
 * round-to-nearest at the end of each chain). Unless opts->bf16_parts says
 * otherwise the passes take three BF16 parts when p < 5 (a nearly square
 * leading block of U^T Omega, whose large inverse amplifies pass rounding;
 * Theorems 1-2) or m n <= 2^27, and two parts above that size, where every
 * entry of a pass sums over K >= ~11600 products and the two-part rounding
 * averages out (measured: |L_ii| within 5e-5 of the FP64 oracle at 16384^2
 * and 20000^2 for sigma_1 / sigma_k up to 100). workspace must be 256-byte
 * aligned and
 * hold rqlp_workspace_bytes(...) bytes; its contents on entry are ignored.
 * d_info: RQLP_INFO_INTS device ints (required). d_diag: RQLP_DIAG_DOUBLES
 * device doubles or NULL. opts may be NULL (defaults). Output buffers must
 * not overlap the inputs or the workspace. */
rqlp_status rqlp_factor(const float* A, int64_t m, int64_t n, int64_t lda,
                        int k, int p, int q,
                        const float* Omega, int64_t ldo,
                        float* Q, int64_t ldq,
                        float* L, int64_t ldl,
                        float* P, int64_t ldp,
                        void* workspace, size_t ws_bytes,
                        int* d_info, double* d_diag,
                        const rqlp_opts* opts, void* stream);

/* Host-buffer form of rqlp_factor: A, Omega, Q, L, P are HOST pointers
 * (pinned memory gives full copy bandwidth). The inputs are copied to the
 * device, factored, and the factors copied back; the call returns after the
 * stream has been synchronised. workspace (device) must hold
 * rqlp_host_workspace_bytes(...) bytes. h_info (2 ints) and h_diag (4
 * doubles, may be NULL) are host arrays with the layouts above. Every return
 * after the first copy has been enqueued (error returns included) follows a
 * synchronisation of the stream, so the host buffers are free for reuse when
 * the call returns. */
size_t rqlp_host_workspace_bytes(int64_t m, int64_t n, int k, int p, int q,
                                 const rqlp_opts* opts);
rqlp_status rqlp_factor_host(const float* hA, int64_t m, int64_t n, int64_t lda,
                             int k, int p, int q,
                             const float* hOmega, int64_t ldo,
                             float* hQ, int64_t ldq,
                             float* hL, int64_t ldl,
                             float* hP, int64_t ldp,
                             void* workspace, size_t ws_bytes,
                             int* h_info, double* h_diag,
                             const rqlp_opts* opts, void* stream);

/* ---- Factorisation without any allocation (the paper has no counterpart;
 * this serves callers of the library, not the method).
 *
 * Some callers cannot allocate device memory: code inside a framework or host
 * application whose own pool owns every byte of device memory, code with a
 * fixed device-memory budget, and code on paths where the implicit device
 * synchronisation of cudaMalloc is not acceptable. rqlp_factor_noalloc is
 * rqlp_factor without the workspace argument: its scratch is one array of
 * RQLP_NOALLOC_SCRATCH_BYTES bytes in device memory that belongs to the
 * library (every GPU that loads the library holds it until the process
 * exits). It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - Problems with rqlp_workspace_bytes(...) > RQLP_NOALLOC_SCRATCH_BYTES
 *    return RQLP_ERR_WORKSPACE and enqueue nothing (16 MiB covers, e.g.,
 *    4096 x 4096 with d = 69 and q = 1).
 *  - All calls on a device share the array, which keeps the last call's
 *    contents; each call clears what must start at zero in its first kernel.
 *    Calls whose GPU work overlaps (two streams without an ordering) race on
 *    the array: order them on one stream or with events.
 *  - The first call on a device looks up the array's device address while
 *    that device is current; make that first call before any stream capture.
 * Other arguments, outputs and errors are as for rqlp_factor. */
#define RQLP_NOALLOC_SCRATCH_BYTES (16u << 20)
rqlp_status rqlp_factor_noalloc(const float* A, int64_t m, int64_t n, int64_t lda,
                                int k, int p, int q,
                                const float* Omega, int64_t ldo,
                                float* Q, int64_t ldq,
                                float* L, int64_t ldl,
                                float* P, int64_t ldp,
                                int* d_info, double* d_diag,
                                const rqlp_opts* opts, void* stream);

/* ---- Step-level entry points (one step of the chain each; same conventions).
 *
 * rqlp_sketch: one pass over A (Algorithm 1 steps 3-4 and each power pass).
 *   trans = 1: Y (n x d, ldy) = A^T X with X m x d (ldx);
 *   trans = 0: Y (m x d, ldy) = A X   with X n x d (ldx).
 *   opts->precision selects FP32 or the BF16x3 tensor-core form. */
size_t rqlp_sketch_workspace_bytes(int trans, int64_t m, int64_t n, int d, const rqlp_opts* opts);
rqlp_status rqlp_sketch(int trans, const float* A, int64_t m, int64_t n, int64_t lda,
                        const float* X, int64_t ldx, int d, float* Y, int64_t ldy,
                        void* workspace, size_t ws_bytes, const rqlp_opts* opts, void* stream);

/* rqlp_orth: X = qf(X) in place, the orth(.) of Algorithm 1 steps 3-4 (thin
 * unpivoted QR, section 2) for a rows x d matrix (rows >= d) by CholeskyQR2,
 * with a diagonal shift and a third pass when a Cholesky breaks down
 * (shifted CholeskyQR3). R (d x d, ldr, may be NULL) receives the upper
 * triangular factor with positive diagonal. d_info as for rqlp_factor. */
size_t rqlp_orth_workspace_bytes(int64_t rows, int d, const rqlp_opts* opts);
rqlp_status rqlp_orth(float* X, int64_t rows, int d, int64_t ldx, float* R, int64_t ldr,
                      void* workspace, size_t ws_bytes, int* d_info, const rqlp_opts* opts,
                      void* stream);

/* ---- Learned (q, p) (no counterpart in the paper, which fixes neither q nor
 * p). A probe sketch Y_w = A^T Omega_w of width w = k + 20 (the widest sketch
 * any p in {5, 10, 20} needs) has its R factor computed (FP32 Gram and
 * Cholesky in both precisions); 12 statistics of its R-diagonal feed a
 * 3-layer MLP (12 -> 64 -> 64 -> 15, ReLU) whose 15 outputs estimate, for
 * every (q, p) with q in {0, 1, 2, 3, 4} and p in {5, 10, 20} (output
 * 3 qi + pi), log10 of the excess rank-k error
 *   eps = ||A - A P_k P_k^T||_F / (sum_{i>k} sigma_i^2)^(1/2) - 1
 * that the chain with that (q, p) reaches. The prediction for a request
 * `target` is the cheapest pair, by cost (2q + 2)(k + p), whose estimate plus
 * the network's calibrated margin delta is at most log10(target) (ties:
 * smaller q, then smaller p); (4, 20) when no pair qualifies. The probe is the
 * first sketch of the chain and its R factor the chain's first
 * orthonormalisation, so prediction costs no extra pass over A. A failed
 * probe (non-zero d_info status) or a non-finite estimate falls back to
 * q = 2, p = 10.
 *
 * Parameters: RQLP_MLP_PARAMS floats, device, layout W1 (12 x 64 row-major),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (64 x 15), b3 (15), delta (1, log10
 * units; set by calibration on held-out data, its gradient is 0). target:
 * 0 < target < 1, else RQLP_ERR_ARG. */
#define RQLP_MLP_FEATURES 12
#define RQLP_MLP_HIDDEN 64
#define RQLP_MLP_OUTPUTS 15
#define RQLP_MLP_PARAMS 5968

/* Forward pass: estimates (batch x 15) of features X (batch x 12), device. */
rqlp_status rqlp_mlp_forward(const float* params, const float* X, int batch, float* est,
                             void* stream);
/* Mean over the batch and the 15 outputs of (estimate - Y)^2 and its gradient
 * (RQLP_MLP_PARAMS floats, 0 for delta) for targets Y (batch x 15, device;
 * log10 of the measured errors). loss: 1 device float (may be NULL).
 * workspace: rqlp_mlp_workspace_bytes(batch) bytes, device. Deterministic
 * (fixed summation order). */
size_t rqlp_mlp_workspace_bytes(int batch);
rqlp_status rqlp_mlp_grad(const float* params, const float* X, const float* Y, int batch,
                          float* grad, float* loss, void* workspace, size_t ws_bytes,
                          void* stream);
/* One Adam step (step is 1-based) on n parameters with moments m1, m2. */
rqlp_status rqlp_mlp_adam(float* params, const float* grad, float* m1, float* m2, int n,
                          float lr, float beta1, float beta2, float eps, int step, void* stream);

/* Probe features (12 device floats) of A (m x n) with Omega (m x (k+20)).
 * Workspace: rqlp_learned_workspace_bytes(...). d_info as for rqlp_factor. */
size_t rqlp_learned_workspace_bytes(int64_t m, int64_t n, int k, const rqlp_opts* opts);
rqlp_status rqlp_probe_features(const float* A, int64_t m, int64_t n, int64_t lda, int k,
                                const float* Omega, int64_t ldo, float* feat,
                                void* workspace, size_t ws_bytes, int* d_info,
                                const rqlp_opts* opts, void* stream);
/* Probe + MLP + selection: d_qp (2 device ints) receives (q, p). */
rqlp_status rqlp_predict_qp(const float* A, int64_t m, int64_t n, int64_t lda, int k,
                            const float* Omega, int64_t ldo, double target, const float* params,
                            int* d_qp, void* workspace, size_t ws_bytes, int* d_info,
                            const rqlp_opts* opts, void* stream);
/* Rand-QLP with the predicted (q, p): the probe is the chain's first sketch
 * (Omega's first k + p columns). Q (m x (k+p)), L, P (n x (k+p)) must have
 * room for k + 20 columns. h_qp (2 host ints) receives the (q, p) used.
 * Synchronises the stream once (to read (q, p)), so it cannot be captured. */
rqlp_status rqlp_factor_learned(const float* A, int64_t m, int64_t n, int64_t lda, int k,
                                const float* Omega, int64_t ldo, double target, const float* params,
                                float* Q, int64_t ldq, float* L, int64_t ldl, float* P, int64_t ldp,
                                void* workspace, size_t ws_bytes, int* d_info, double* d_diag,
                                int* h_qp, const rqlp_opts* opts, void* stream);

/* Host-buffer form of rqlp_factor_learned: A (m x n, lda), Omega
 * (m x (k+20), ldo), Q, L, P are HOST pointers (pinned memory gives full copy
 * bandwidth; params stays a device pointer). A and Omega are copied to the
 * device by row blocks on two copy streams that the library owns (created on
 * the first call on each device), and each block's share of the probe
 * sketch, A_b^T Omega_b, starts as soon as the block has landed, so the copy
 * of A overlaps its first pass over A; the shares are summed in FP32 in
 * block order (the sketch can therefore differ from rqlp_factor_learned's in
 * the last bits). Then features, (q, p) (read back: one synchronisation), the
 * chain, and the factors' copy back; returns after the stream has been
 * synchronised, error returns included. Calls on one device are serialised.
 * workspace (device) must hold rqlp_learned_host_workspace_bytes(...) bytes;
 * h_info (2 ints), h_diag (4 doubles, may be NULL) and h_qp (2 ints) are host
 * arrays. Q, L, P receive k + p columns (their buffers need room for k + 20).
 * The copy/compute overlap is this library's; the factorisation is
 * Algorithm 1 as in rqlp_factor_learned. */
size_t rqlp_learned_host_workspace_bytes(int64_t m, int64_t n, int k, const rqlp_opts* opts);
rqlp_status rqlp_factor_learned_host(const float* hA, int64_t m, int64_t n, int64_t lda, int k,
                                     const float* hOmega, int64_t ldo, double target,
                                     const float* params, float* hQ, int64_t ldq,
                                     float* hL, int64_t ldl, float* hP, int64_t ldp,
                                     void* workspace, size_t ws_bytes, int* h_info,
                                     double* h_diag, int* h_qp, const rqlp_opts* opts,
                                     void* stream);

/* ---- Batched form: many independent problems, each with its own sizes,
 * k, p and buffers (one q for the batch), factored by the chain of
 * rqlp_factor. opts->precision: RQLP_PREC_FP32 (every product in FP32), or
 * RQLP_PREC_BF16X3: the passes over A run as grouped tensor-core passes over
 * BF16 halves of every A (split once per launch into the workspace, which
 * then also holds the halves, the pass operands' halves and eight tensor
 * maps per problem), the d-wide products in FP32; RQLP_ERR_UNSUPPORTED on a
 * device without the tensor-core path. The passes take three BF16 parts per
 * operand (six products, FP32-level rounding) unless opts->bf16_parts = 2
 * (three products, ~2^-16 of |A| |X| per pass).
 *
 * A batch plan is built once on the host: it lays out the caller's
 * workspace, writes the per-problem job tables into it (one synchronous
 * copy on `stream` at creation) and fixes the launch sequence. Each step of
 * the chain is one grouped launch over all problems; rqlp_batch_launch
 * captures the sequence into a CUDA graph on first use and replays it as
 * one launch (stream-ordered, no host synchronisation). The plan is bound to
 * the buffers it was created with; the problems' matrices may change
 * between launches, their addresses and sizes may not.
 *
 * Problems: A (m x n, lda >= n), Omega (m x (k+p), ldo >= k+p), outputs as
 * in rqlp_factor; 1 <= k, p >= 0, d = k + p <= min(m, n) and
 * d <= RQLP_BATCH_MAX_D, else RQLP_ERR_ARG. d_info: 2 device ints per
 * problem (caller's order), d_diag: 4 device doubles per problem (optional),
 * laid out as for rqlp_factor.
 *
 * rqlp_batch_autotune times every tile configuration (6 tile shapes x
 * persistent or one-CTA-per-tile grids) of each grouped product shape (tall
 * A^T X, tall A X, Gram, X R^{-1}, d x d) and width bucket (d <= 32, d > 32)
 * on the plan's own problems, keeps the fastest and
 * remembers the choice for later plans with the same size mix (process
 * wide). It runs products out of order on the workspace: run it before the
 * batch is launched, then launch. rqlp_batch_tuning writes the chosen
 * configuration ids (shape-major, 2 buckets per shape; id = tile shape 0..5,
 * plus 6 for one CTA per tile) and returns their count. In the BF16X3 form
 * the tall shapes' ids are unused (those passes run on the tensor cores). */
#define RQLP_BATCH_MAX_D 128
typedef struct {
  const float* A; int64_t m, n, lda;
  const float* Omega; int64_t ldo;
  int k, p;
  float* Q; int64_t ldq;
  float* L; int64_t ldl;
  float* P; int64_t ldp;
} rqlp_problem;
typedef struct rqlp_batch_s* rqlp_batch;

size_t rqlp_batch_workspace_bytes(int count, const rqlp_problem* probs, int q, const rqlp_opts* opts);
rqlp_status rqlp_batch_create(int count, const rqlp_problem* probs, int q, void* workspace,
                              size_t ws_bytes, int* d_info, double* d_diag, const rqlp_opts* opts,
                              void* stream, rqlp_batch* out);
rqlp_status rqlp_batch_autotune(rqlp_batch batch, int reps, void* stream);
int rqlp_batch_tuning(rqlp_batch batch, int* cfg, int cap);
/* Plain launches of the whole sequence (no graph). */
rqlp_status rqlp_batch_run(rqlp_batch batch, void* stream);
/* The sequence as one graph launch (captured on first use). */
rqlp_status rqlp_batch_launch(rqlp_batch batch, void* stream);
rqlp_status rqlp_batch_destroy(rqlp_batch batch);
/* create + launch + synchronise + destroy. */
rqlp_status rqlp_factor_batched(int count, const rqlp_problem* probs, int q, void* workspace,
                                size_t ws_bytes, int* d_info, double* d_diag, const rqlp_opts* opts,
                                void* stream);

/* ---- Sparse A (section 5.1 factors sparse matrices; Algorithm 1 touches A
 * only through products with A and A^T).
 *
 * rqlp_factor_sparse: the chain of rqlp_factor for A in CSR form (device
 * arrays: row_ptr (m + 1 int64, row_ptr[0] = 0, non-decreasing, row_ptr[m] =
 * nnz), col_idx (nnz int32 in [0, n)), vals (nnz float)); the passes over A
 * are sparse-times-dense products (a warp per row, the nonzeros of a row in
 * storage order, FP32), and A^T is built on the device in CSR form at the
 * start of every call (column counts, scan, scatter, each column sorted by
 * row: every sum runs in a fixed order). Other arguments, outputs and
 * errors as for rqlp_factor; FP32 only (opts->precision = RQLP_PREC_FP32,
 * else RQLP_ERR_UNSUPPORTED: the products are gathers, not dense
 * contractions), step 5 on the d x d R. A column index outside [0, n) or a
 * decreasing row pointer is skipped and reported as RQLP_ERR_ARG in d_info.
 * workspace: rqlp_sparse_workspace_bytes(A, k, p, q, opts) bytes, 256-byte
 * aligned (the chain's workspace plus A^T: 8 (n + 1) + 8 nnz + 4 n bytes). */
typedef struct {
  int64_t m, n, nnz;
  const int64_t* row_ptr;
  const int* col_idx;
  const float* vals;
} rqlp_csr;
size_t rqlp_sparse_workspace_bytes(const rqlp_csr* A, int k, int p, int q, const rqlp_opts* opts);
rqlp_status rqlp_factor_sparse(const rqlp_csr* A, int k, int p, int q,
                               const float* Omega, int64_t ldo,
                               float* Q, int64_t ldq, float* L, int64_t ldl, float* P, int64_t ldp,
                               void* workspace, size_t ws_bytes, int* d_info, double* d_diag,
                               const rqlp_opts* opts, void* stream);

/* ---- Evaluation utilities on the device (section 5.2: rank-r
 * approximations; section 4.1, Theorem 2: distances between subspaces).
 *
 * rqlp_rank_errors: errs[r - 1] = ||A - A_r||_F for r = 1..d, where
 *   A_r = Q L(:, 1:r) P(:, 1:r)^T, from the factors of rqlp_factor: this
 *   chain's A_r is A P_r P_r^T (Q L P^T = A P~ P~^T), so ||A - A_r||_F^2 =
 *   ||A||_F^2 - ||L(:, 1:r)||_F^2 with ||A||_F^2 = d_diag[0] (device, from
 *   rqlp_factor). L (d x d, device, ldl), errs: d device doubles.
 * rqlp_rank_residual: *out = ||A - Q L(:, 1:r) P(:, 1:r)^T||_F computed
 *   explicitly (one pass over A, FP32 products, FP64 sums; 1 device double),
 *   for checking the identity or factors that did not come from this chain.
 *   workspace: rqlp_rank_residual_workspace_bytes(m, r), 256-byte aligned.
 * rqlp_subspace_angles: for orthonormal X (rows x a, ldx) and Y (rows x b,
 *   ldy), device, out (b device doubles, largest first) receives the sines
 *   of the canonical angles between R(Y) and R(X) -- the singular values of
 *   (I - X X^T) Y; out[0] is the distance sin theta of Theorem 2 when a = b
 *   -- or, with cosines = 1, the singular values of X^T Y (out[0] =
 *   ||X^T Y||_2, the form of the sin phi bounds with Y the trailing columns
 *   of Q or P). The b x b Gram of that matrix is formed in FP64 and its
 *   eigenvalues found by cyclic Jacobi on one CTA (a check, not a fast path):
 *   sines resolve down to ~1e-7 of FP32 input. workspace:
 *   rqlp_subspace_workspace_bytes(rows, a, b), 256-byte aligned.
 * All three are stream-ordered; sizes out of range return RQLP_ERR_ARG. */
rqlp_status rqlp_rank_errors(const float* L, int64_t ldl, int d, const double* d_diag, double* errs,
                             void* stream);
size_t rqlp_rank_residual_workspace_bytes(int64_t m, int r);
rqlp_status rqlp_rank_residual(const float* A, int64_t m, int64_t n, int64_t lda,
                               const float* Q, int64_t ldq, const float* L, int64_t ldl, int d,
                               const float* P, int64_t ldp, int r, double* out,
                               void* workspace, size_t ws_bytes, void* stream);
size_t rqlp_subspace_workspace_bytes(int64_t rows, int a, int b);
rqlp_status rqlp_subspace_angles(const float* X, int64_t rows, int a, int64_t ldx,
                                 const float* Y, int b, int64_t ldy, int cosines, double* out,
                                 void* workspace, size_t ws_bytes, void* stream);

/* ---- Runtime services (host only; no device memory).
 *
 * rqlp_kernel_launches: cumulative number of CUDA kernels this library has
 * launched in the calling process.
 * rqlp_profile_enable(on): while on, every pass over A (the dense products
 * A^T X and A X) is bracketed by a CUDA event pair recorded on the launching
 * stream. Returns the previous state. Do not enable it while capturing a
 * graph.
 * rqlp_profile_read: after synchronising the stream, writes up to cap pass
 * durations in ms (tags[i] = 1 for A^T X, 0 for A X) in launch order, clears
 * the record list and returns the count written. */
unsigned long long rqlp_kernel_launches(void);
int rqlp_profile_enable(int on);
int rqlp_profile_read(float* ms, int* tags, int cap);

/* Human-readable name of a status code (static string). */
const char* rqlp_status_string(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int rqlp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RQLP_H */
