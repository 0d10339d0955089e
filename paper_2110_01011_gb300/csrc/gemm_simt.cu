// FP32 SIMT GEMM engine: the plain-FP32 passes over A (Y = A^T X, Z = A X,
// Algorithm 1 steps 3-4 and the power passes) and the tall-skinny products of
// CholeskyQR (Gram X^T X, X R^{-1}).
//
// C = op(A) B with op(A) = A^T (transA) or A, row-major operands. Each CTA
// owns a BM x BN tile of C and one slice of the K range (split-K); slices
// write partial tiles that a second kernel sums in a fixed order (Kahan), so
// results are deterministic. Tiles reach shared memory by asynchronous copies
// (cp.async) through a ring of three or four stages, so a CTA pays the global
// latency about once per K range rather than once per 16-wide K tile (the
// d x d products of CholeskyQR have K = d and only a handful of tiles); each
// thread accumulates a TM x TN block in registers.
#include <algorithm>

#include "common.cuh"

namespace rqlp {

namespace {

struct GemmArgs {
  int64_t M, N, K;
  const float* A; int64_t lda;
  const float* B; int64_t ldb;
  float* C; int64_t ldc; int64_t c_slice;   // slice z writes C + z * c_slice
  int64_t kchunk;                           // K range per slice (multiple of BK)
  double* sumsq;                            // optional sum of squares of A
  const int* gate;                          // optional gate word (see GateMode)
  int gate_mode;
  int b_upper;                              // B upper triangular: skip k >= n-tile end
  int lower_only;                           // only tiles with entries on or below the diagonal
};

// Gated off (kGateCopy): C = A on this tile (B taken as the identity). All
// loads of the thread are issued before its stores (C and A are distinct
// buffers, which the compiler cannot assume), four 128-bit loads at a time.
template <int BM, int BN, int NT>
__device__ __forceinline__ void copy_tile(const GemmArgs& g, int64_t m0, int64_t n0, float* C) {
  constexpr int Q = BN / 4;            // float4 per tile row
  constexpr int PER = BM * Q / NT;     // float4 per thread
  constexpr int CH = 4;                // float4 loaded before their stores (bounded registers)
  static_assert(PER * NT == BM * Q, "copy tiling");
  const bool vec = ((reinterpret_cast<uintptr_t>(g.A) | reinterpret_cast<uintptr_t>(C)) % 16 == 0) &&
                   g.lda % 4 == 0 && g.ldc % 4 == 0;
#pragma unroll 1
  for (int r0 = 0; r0 < PER; r0 += CH) {
    float4 v[CH];
#pragma unroll
    for (int r = 0; r < CH; ++r) {
      if (r0 + r >= PER) break;
      const int f = threadIdx.x + (r0 + r) * NT;
      const int64_t gm = m0 + f / Q, gn = n0 + (f % Q) * 4;
      const float* src = g.A + gm * g.lda + gn;
      if (gm < g.M && vec && gn + 3 < g.N) {
        v[r] = *reinterpret_cast<const float4*>(src);
      } else {
        float t[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = (gm < g.M && gn + i < g.N) ? src[i] : 0.f;
        v[r] = make_float4(t[0], t[1], t[2], t[3]);
      }
    }
#pragma unroll
    for (int r = 0; r < CH; ++r) {
      if (r0 + r >= PER) break;
      const int f = threadIdx.x + (r0 + r) * NT;
      const int64_t gm = m0 + f / Q, gn = n0 + (f % Q) * 4;
      if (gm >= g.M) continue;
      float* dst = C + gm * g.ldc + gn;
      if (vec && gn + 3 < g.N) {
        *reinterpret_cast<float4*>(dst) = v[r];
      } else {
        const float t[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (gn + i < g.N) dst[i] = t[i];
      }
    }
  }
}

// One BM x BN tile of C (rows m0.., columns n0..) over K-slice `slice`, by the
// whole CTA.
// FAST_COPY: the gated copy by copy_tile (single-matrix kernels); the
// grouped kernels keep a plain per-element loop, which holds no registers
// beyond the main loop's (copy_tile raises their spills at 128 registers).
template <int BM, int BN, int BK, int TM, int TN, bool TRANS_A, bool FAST_COPY = true>
__device__ __forceinline__ void gemm_tile(const GemmArgs& g, int64_t m0, int64_t n0, int slice) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  constexpr int AL = BM * BK / NT;
  constexpr int BL = BN * BK / NT;
  constexpr int QA = BM / 4, QB = BN / 4;          // 16-byte chunks per tile row
  constexpr int AV = BK * QA / NT, BV = BK * QB / NT;
  static_assert(AL * NT == BM * BK && BL * NT == BN * BK, "tile/thread mismatch");
  static_assert(AV * NT == BK * QA && BV * NT == BK * QB, "chunk/thread mismatch");
  constexpr int S = BM * BN <= 2048 ? 4 : 3;       // stages in the ring
  __shared__ __align__(16) float As[S][BK][BM + 4];
  __shared__ __align__(16) float Bs[S][BK][BN + 4];

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  float* C = g.C + (int64_t)slice * g.c_slice;
  if (g.lower_only && n0 > m0 + BM - 1) return;   // every entry of the tile has j > i

  if (g.gate != nullptr && *g.gate == 0) {
    if (g.gate_mode == kGateSkip) return;
    // Gated off: B is taken as the identity (requires !TRANS_A, K == N, one slice).
    if (FAST_COPY) {
      copy_tile<BM, BN, NT>(g, m0, n0, C);
    } else {
      for (int idx = tid; idx < BM * BN; idx += NT) {
        const int64_t gm = m0 + idx / BN, gn = n0 + idx % BN;
        if (gm < g.M && gn < g.N) C[gm * g.ldc + gn] = g.A[gm * g.lda + gn];
      }
    }
    return;
  }

  const int64_t kbeg = (int64_t)slice * g.kchunk;
  int64_t kend = kbeg + g.kchunk < g.K ? kbeg + g.kchunk : g.K;
  if (g.b_upper && kend > n0 + BN) kend = n0 + BN;
  const int64_t ntiles = kend > kbeg ? cdiv(kend - kbeg, BK) : 0;

  float sq = 0.f, sq_c = 0.f;   // Kahan sum of squares of the A tiles read
  const bool want_sq = g.sumsq != nullptr && n0 == 0;   // each element of A once

  // A tile: As[kk][mm] = op(A)(m0 + mm, k0 + kk); B tile: Bs[kk][nn] =
  // B(k0 + kk, n0 + nn); zeros outside [0, M) x [k0, kend) x [0, N). A smem
  // row that is contiguous in global memory (B's rows; A^T's rows) goes as
  // 16-byte chunks when the operand is 16-byte aligned with a row stride that
  // is a multiple of 4; A (not transposed) is transposed element by element.
  const bool vecA = TRANS_A && (reinterpret_cast<uintptr_t>(g.A) & 15) == 0 && (g.lda & 3) == 0;
  const bool vecB = (reinterpret_cast<uintptr_t>(g.B) & 15) == 0 && (g.ldb & 3) == 0;
  auto issue = [&](int64_t k0, int buf) {
    if (vecA) {
#pragma unroll
      for (int r = 0; r < AV; ++r) {
        const int idx = tid + r * NT, kk = idx / QA, mq = idx % QA;
        const int64_t gk = k0 + kk, gm = m0 + 4 * mq;
        const int64_t left = g.M - gm;
        const int valid = gk < kend && left > 0 ? (left < 4 ? (int)left : 4) : 0;
        cp_async16(&As[buf][kk][4 * mq], valid > 0 ? g.A + gk * g.lda + gm : g.A, 4 * valid);
      }
    } else {
#pragma unroll
      for (int r = 0; r < AL; ++r) {
        const int idx = tid + r * NT;
        const int kk = TRANS_A ? idx / BM : idx % BK;
        const int mm = TRANS_A ? idx % BM : idx / BK;
        const int64_t gk = k0 + kk, gm = m0 + mm;
        const bool ok = gk < kend && gm < g.M;
        const float* src = !ok ? g.A : (TRANS_A ? g.A + gk * g.lda + gm : g.A + gm * g.lda + gk);
        cp_async4(&As[buf][kk][mm], src, ok ? 4 : 0);
      }
    }
    if (vecB) {
#pragma unroll
      for (int r = 0; r < BV; ++r) {
        const int idx = tid + r * NT, kk = idx / QB, nq = idx % QB;
        const int64_t gk = k0 + kk, gn = n0 + 4 * nq;
        const int64_t left = g.N - gn;
        const int valid = gk < kend && left > 0 ? (left < 4 ? (int)left : 4) : 0;
        cp_async16(&Bs[buf][kk][4 * nq], valid > 0 ? g.B + gk * g.ldb + gn : g.B, 4 * valid);
      }
    } else {
#pragma unroll
      for (int r = 0; r < BL; ++r) {
        const int idx = tid + r * NT, kk = idx / BN, nn = idx % BN;
        const int64_t gk = k0 + kk, gn = n0 + nn;
        const bool ok = gk < kend && gn < g.N;
        cp_async4(&Bs[buf][kk][nn], ok ? g.B + gk * g.ldb + gn : g.B, ok ? 4 : 0);
      }
    }
  };
  // Squares of the A entries this thread copied into stage buf (zeros past
  // the edges), Kahan-summed.
  auto add_squares = [&](int buf) {
    float sacc = 0.f;
    if (vecA) {
#pragma unroll
      for (int r = 0; r < AV; ++r) {
        const int idx = tid + r * NT, kk = idx / QA, mq = idx % QA;
        const float4 v = *reinterpret_cast<const float4*>(&As[buf][kk][4 * mq]);
        sacc = fmaf(v.x, v.x, sacc); sacc = fmaf(v.y, v.y, sacc);
        sacc = fmaf(v.z, v.z, sacc); sacc = fmaf(v.w, v.w, sacc);
      }
    } else {
#pragma unroll
      for (int r = 0; r < AL; ++r) {
        const int idx = tid + r * NT;
        const int kk = TRANS_A ? idx / BM : idx % BK;
        const int mm = TRANS_A ? idx % BM : idx / BK;
        const float v = As[buf][kk][mm];
        sacc = fmaf(v, v, sacc);
      }
    }
    const float y = sacc - sq_c, t = sq + y;
    sq_c = (t - sq) - y;
    sq = t;
  };

  // Two-level accumulation: acc runs over kPromoteTiles K-tiles (256 of K)
  // and is then added into tot, so the rounding of a long K range grows with
  // 256 + K / 256 terms instead of K (the Gram of a 4000-row block lost an
  // order of magnitude of orthogonality to one running sum).
  constexpr int kPromoteTiles = 256 / BK;
  float acc[TM][TN], tot[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = tot[i][j] = 0.f;

  if (ntiles > 0) {
    // Ring: tile t lives in stage t % S; S - 1 tiles are in flight ahead of
    // the one being multiplied. The barrier at the top of iteration t also
    // ends every thread's reads of stage (t - 1) % S, which iteration t refills.
#pragma unroll
    for (int st = 0; st < S - 1; ++st) {
      if (st < ntiles) issue(kbeg + st * BK, st);
      cp_async_commit();
    }
    for (int64_t t = 0; t < ntiles; ++t) {
      const int buf = (int)(t % S);
      cp_async_wait<S - 2>();   // this thread's copies of tile t have landed
      __syncthreads();
      if (t + S - 1 < ntiles) issue(kbeg + (t + S - 1) * BK, (int)((t + S - 1) % S));
      cp_async_commit();
      if (want_sq) add_squares(buf);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; i += 4) {
          float4 v = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM + i]);
          a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
        }
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
          float4 v = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * TN + j]);
          b[j] = v.x; b[j + 1] = v.y; b[j + 2] = v.z; b[j + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if ((t + 1) % kPromoteTiles == 0) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            tot[i][j] += acc[i][j];
            acc[i][j] = 0.f;
          }
      }
    }
    cp_async_wait_all();   // only empty groups can remain; the stages are free
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] += tot[i][j];

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gm = m0 + ty * TM + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t gn = n0 + tx * TN + j;
      if (gn < g.N) C[gm * g.ldc + gn] = acc[i][j];
    }
  }

  if (want_sq) {
    // Block reduction of the per-thread sums in double, one atomic per CTA.
    __shared__ double red[32];
    double v = (double)sq - (double)sq_c;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      atomicAdd(g.sumsq, s);
    }
  }
}

// Registers: 512 threads' worth per CTA count, as in the grouped form (at
// most 128 per thread).
template <int BM, int BN, int BK, int TM, int TN, bool TRANS_A>
__global__ void __launch_bounds__((BM / TM) * (BN / TN), 512 / ((BM / TM) * (BN / TN)))
gemm_f32_kernel(GemmArgs g) {
  gemm_tile<BM, BN, BK, TM, TN, TRANS_A>(g, (int64_t)blockIdx.y * BM, (int64_t)blockIdx.x * BN, blockIdx.z);
}

// Grouped form: the tiles of every problem's C in one list (tile_start is the
// exclusive prefix sum of the per-problem tile counts); persistent CTAs walk
// the list. Problem b's tiles run over its M x N output in row-major order.
// Registers: 512 threads' worth per CTA count (four 128-thread CTAs per SM);
// measured faster on the bench batch than a 384-thread cap without spills
// (30.3 vs 31.9 ms for the FP32 form).
template <int BM, int BN, int BK, int TM, int TN, bool TRANS_A>
__global__ void __launch_bounds__((BM / TM) * (BN / TN), 512 / ((BM / TM) * (BN / TN)))
gemm_grouped_kernel(const GroupGemm* __restrict__ jobs, const int* __restrict__ tile_start, int count) {
  const int total = tile_start[count];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = count - 1;   // last b with tile_start[b] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_start[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const GroupGemm& j = jobs[lo];
    const int local = t - tile_start[lo];
    const int tn = (int)cdiv(j.N, BN);
    GemmArgs g;
    g.M = j.M; g.N = j.N; g.K = j.K;
    g.A = j.A; g.lda = j.lda;
    g.B = j.B; g.ldb = j.ldb;
    g.C = j.C; g.ldc = j.ldc; g.c_slice = 0;
    g.kchunk = round_up(j.K > 0 ? j.K : 1, BK);
    g.sumsq = j.sumsq;
    g.gate = j.gate;
    g.gate_mode = j.gate_mode;
    g.b_upper = j.b_upper;
    g.lower_only = j.lower_only;
    __syncthreads();   // the previous tile's shared-memory reads are done
    gemm_tile<BM, BN, BK, TM, TN, TRANS_A, false>(g, (int64_t)(local / tn) * BM, (int64_t)(local % tn) * BN, 0);
  }
}

// Wide tile for the passes over A and the tall products with N >= 96: one
// 128 x BN tile of C per CTA of 256 threads, 8 x (4 + TN2) outputs per thread
// in two 4-wide row groups (ty * 4 .., 64 + ty * 4 ..) and two column groups
// (tx * 4 .. + 3 and 64 + tx * TN2 .., TN2 = (BN - 64) / 16), so that four
// conflict-free 128-bit shared loads feed 64 FMAs at BN = 128 (the 128 x 64
// tile needs three per 32). BN = 112 (TN2 = 3, the second group read by three
// conflict-free 32-bit loads) covers N = 210 in 224 columns instead of 256.
// VEC: A and B are 16-byte aligned with row strides that are multiples of 4
// floats, and tiles are fetched with 128-bit global loads. Same K slicing,
// gates, sum of squares and two-level accumulation as gemm_tile; the second
// level (8 x TN per thread) lives in dynamic shared memory, so that a thread
// fits in 128 registers and two CTAs share an SM.
constexpr int kWideBM = 128, kWideBK = 16, kWideThreads = 256, kWidePerSm = 2;
template <int BN>
constexpr size_t wide_tot_bytes() { return (size_t)8 * (4 + (BN - 64) / 16) * kWideThreads * sizeof(float); }

template <bool TRANS_A, bool VEC, int BN>
__global__ void __launch_bounds__(kWideThreads, kWidePerSm) gemm_f32_wide_kernel(GemmArgs g) {
  constexpr int BM = kWideBM, BK = kWideBK, NT = kWideThreads;
  constexpr int TN2 = (BN - 64) / 16, TN = 4 + TN2;
  constexpr int QB = BN / 4;                 // float4 per row of a B tile
  static_assert(BN == 112 || BN == 128, "wide tile widths");
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int slice = blockIdx.z;
  float* C = g.C + (int64_t)slice * g.c_slice;

  if (g.gate != nullptr && *g.gate == 0) {
    if (g.gate_mode == kGateSkip) return;
    copy_tile<BM, BN, NT>(g, m0, n0, C);   // B taken as the identity (see gemm_tile)
    return;
  }

  const int64_t kbeg = (int64_t)slice * g.kchunk;
  int64_t kend = kbeg + g.kchunk < g.K ? kbeg + g.kchunk : g.K;
  if (g.b_upper && kend > n0 + BN) kend = n0 + BN;
  const int64_t ntiles = kend > kbeg ? cdiv(kend - kbeg, BK) : 0;
  const bool want_sq = g.sumsq != nullptr && n0 == 0;
  float sq = 0.f, sq_c = 0.f;

  // Per thread and K tile: two float4 of A and two of B (512 of each per tile).
  float4 ra[2], rb[2];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int f = tid + r * NT;
      float v[4];
      if (TRANS_A) {   // A stored K x M: tile row kk, columns mq * 4 .. + 3
        const int kk = f / 32, mq = f % 32;
        const int64_t gk = k0 + kk, gm = m0 + mq * 4;
        const float* src = g.A + gk * g.lda + gm;
        if (VEC && gk < kend && gm + 3 < g.M) {
          const float4 t = *reinterpret_cast<const float4*>(src);
          v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = (gk < kend && gm + i < g.M) ? src[i] : 0.f;
        }
      } else {         // A stored M x K: row, k columns kq * 4 .. + 3
        const int row = f / 4, kq = f % 4;
        const int64_t gm = m0 + row, gk = k0 + kq * 4;
        const float* src = g.A + gm * g.lda + gk;
        if (VEC && gm < g.M && gk + 3 < kend) {
          const float4 t = *reinterpret_cast<const float4*>(src);
          v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = (gm < g.M && gk + i < kend) ? src[i] : 0.f;
        }
      }
      ra[r] = make_float4(v[0], v[1], v[2], v[3]);
      if (f < BK * QB) {
        const int kk = f / QB, nq = f % QB;
        const int64_t gk = k0 + kk, gn = n0 + nq * 4;
        const float* src = g.B + gk * g.ldb + gn;
        float w[4];
        if (VEC && gk < kend && gn + 3 < g.N) {
          const float4 t = *reinterpret_cast<const float4*>(src);
          w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) w[i] = (gk < kend && gn + i < g.N) ? src[i] : 0.f;
        }
        rb[r] = make_float4(w[0], w[1], w[2], w[3]);
      }
    }
    if (want_sq) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        s = fmaf(ra[r].x, ra[r].x, s); s = fmaf(ra[r].y, ra[r].y, s);
        s = fmaf(ra[r].z, ra[r].z, s); s = fmaf(ra[r].w, ra[r].w, s);
      }
      const float y = s - sq_c, t = sq + y;
      sq_c = (t - sq) - y;
      sq = t;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int f = tid + r * NT;
      if (TRANS_A) {
        *reinterpret_cast<float4*>(&As[buf][f / 32][(f % 32) * 4]) = ra[r];
      } else {
        const int row = f / 4, k = (f % 4) * 4;
        As[buf][k][row] = ra[r].x; As[buf][k + 1][row] = ra[r].y;
        As[buf][k + 2][row] = ra[r].z; As[buf][k + 3][row] = ra[r].w;
      }
      if (f < BK * QB) *reinterpret_cast<float4*>(&Bs[buf][f / QB][(f % QB) * 4]) = rb[r];
    }
  };

  constexpr int kPromoteTiles = 256 / BK;
  extern __shared__ __align__(16) float tot_s[];   // [8][TN][NT]: entry (i, j) of thread tid
  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[i][j] = 0.f;
      tot_s[(i * TN + j) * NT + tid] = 0.f;
    }

  if (ntiles > 0) {
    load(kbeg);
    store(0);
    __syncthreads();
    for (int64_t t = 0; t < ntiles; ++t) {
      const int buf = (int)(t & 1);
      if (t + 1 < ntiles) load(kbeg + (t + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        float b[TN] = {b0.x, b0.y, b0.z, b0.w};
        if (TN2 == 4) {
          const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
          b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[TN - 1] = b1.w;
        } else {
#pragma unroll
          for (int j = 0; j < TN2; ++j) b[4 + j] = Bs[buf][kk][64 + tx * TN2 + j];
        }
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (t + 1 < ntiles) store(buf ^ 1);
      if ((t + 1) % kPromoteTiles == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            tot_s[(i * TN + j) * NT + tid] += acc[i][j];
            acc[i][j] = 0.f;
          }
      }
      __syncthreads();
    }
  }

  const bool cvec = (reinterpret_cast<uintptr_t>(C) % 16 == 0) && (g.ldc % 4 == 0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gm >= g.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int w = h == 0 ? 4 : TN2;   // columns of this group
      const int64_t gn = n0 + (h == 0 ? tx * 4 : 64 + tx * TN2);
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = j < w ? acc[i][h * 4 + j] + tot_s[(i * TN + h * 4 + j) * NT + tid] : 0.f;
      float* dst = C + gm * g.ldc + gn;
      if (w == 4 && cvec && gn + 3 < g.N) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < w && gn + j < g.N) dst[j] = v[j];
      }
    }
  }

  if (want_sq) {
    __shared__ double red[NT / 32];
    double v = (double)sq - (double)sq_c;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      atomicAdd(g.sumsq, s);
    }
  }
}

// C[m, n] = sum_z part[z][m][n] (fixed order, Kahan-compensated FP32); the
// slices' values are loaded four at a time ahead of the sums. lower_only:
// entries above the diagonal are not summed (the caller reads the lower
// triangle; their partial tiles were never written). A product gated off
// with kGateSkip wrote no partial tiles, and nothing is summed.
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int splits, const float* __restrict__ part,
                                     float* __restrict__ C, int64_t ldc, int lower_only, const int* skip_gate) {
  if (skip_gate != nullptr && *skip_gate == 0) return;
  const int64_t total = M * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / N, col = i % N;
    if (lower_only && col > row) continue;
    float s = 0.f, c = 0.f;
    int z = 0;
    for (; z + 4 <= splits; z += 4) {
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = part[(int64_t)(z + j) * total + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float y = v[j] - c, t = s + y;
        c = (t - s) - y;
        s = t;
      }
    }
    for (; z < splits; ++z) {
      const float y = part[(int64_t)z * total + i] - c, t = s + y;
      c = (t - s) - y;
      s = t;
    }
    C[row * ldc + col] = s;
  }
}

// Tile configuration: the wide 128 x 128 (or 128 x 112) tile, two CTAs per
// SM, for the passes over A of width N >= 96; a 128 x 64 tile (two CTAs per
// SM) or 128 x 32 tile (four) for narrower passes and for the tall products
// with a short K (X R^{-1}, P~ P^: K = d, too few k-tiles for the wide
// tile's deep K loop); a small 32 x 32 tile (eight) for the Grams and d x d
// work.
bool use_wide(int64_t M, int64_t N, int64_t K) { return M >= 1024 && N >= 96 && K >= 1024; }
// Column tile of the wide kernel: 112 where it pads N less than 128 does.
int wide_bn(int64_t N) { return cdiv(N, 112) * 112 < cdiv(N, 128) * 128 ? 112 : 128; }
bool use_big(int64_t M, int64_t N) { return M >= 1024 && N >= 48; }
// Column tile of the large tile: 32 where it pads N less than 64 does and K
// is short (the d-wide products X R^{-1}, P~ P^ with K = d: more, smaller
// CTAs also fill the last wave better); 64 otherwise (a long-K pass reads
// its A once per column tile).
int big_bn(int64_t N, int64_t K) { return K <= 256 && cdiv(N, 32) * 32 < cdiv(N, 64) * 64 ? 32 : 64; }

}  // namespace

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      cached = n;
    else
      cached = 152;
  }
  return cached;
}

int gemm_f32_splits(int64_t M, int64_t N, int64_t K) {
  const bool wide = use_wide(M, N, K), big = use_big(M, N);
  const int64_t BM = big ? 128 : 32, BN = wide ? wide_bn(N) : big ? big_bn(N, K) : 32;
  const int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
  if (wide) {
    // kWidePerSm CTAs per SM: the fewest K slices (1..8, >= 512 of K per
    // slice) whose CTAs fill at least 90 % of their waves, else the fullest.
    const int64_t nsm = (int64_t)sm_count() * kWidePerSm;
    int best = 1;
    double best_eff = 0.0;
    for (int s = 1; s <= 8 && (s == 1 || K / s >= 512); ++s) {
      const int64_t ctas = tiles * s;
      const double eff = (double)ctas / (double)(cdiv(ctas, nsm) * nsm);
      if (eff > best_eff) {
        best_eff = eff;
        best = s;
      }
      if (eff >= 0.9) break;
    }
    return best;
  }
  const int64_t resident = (int64_t)sm_count() * (512 / ((BM / (big ? 8 : 4)) * (BN / 4)));   // CTAs per SM
  int64_t s = cdiv(resident * 2, tiles);            // about two waves of CTAs
  // keep >= 256 K per slice on the large tile; the d x d products of the
  // small tile (K = d) split down to 64 K per slice, as they would otherwise
  // run 49 CTAs at d = 210
  int64_t maxs = big ? K / 256 : K / 64;
  if (s > maxs) s = maxs;
  if (s > 64) s = 64;
  if (s < 1) s = 1;
  return (int)s;
}

size_t gemm_f32_part_floats(int64_t M, int64_t N, int64_t K) {
  int s = gemm_f32_splits(M, N, K);
  return s > 1 ? (size_t)s * (size_t)(M * N) : 0;
}

static cudaError_t launch_gemm(bool transA, const GemmArgs& g, int splits, cudaStream_t st) {
  const bool big = use_big(g.M, g.N);
  if (use_wide(g.M, g.N, g.K)) {
    const bool vec = reinterpret_cast<uintptr_t>(g.A) % 16 == 0 && reinterpret_cast<uintptr_t>(g.B) % 16 == 0 &&
                     g.lda % 4 == 0 && g.ldb % 4 == 0;
    const int bn = wide_bn(g.N);
    dim3 grid((unsigned)cdiv(g.N, bn), (unsigned)cdiv(g.M, kWideBM), (unsigned)splits);
#define RQLP_WIDE(T, V, W)                                                                              \
  do {                                                                                                  \
    static bool set_ = false;                                                                           \
    if (!set_) {                                                                                        \
      const cudaError_t e_ = cudaFuncSetAttribute(gemm_f32_wide_kernel<T, V, W>,                       \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                                  (int)wide_tot_bytes<W>());                            \
      if (e_ != cudaSuccess) return e_;                                                                 \
      set_ = true;                                                                                      \
    }                                                                                                   \
    gemm_f32_wide_kernel<T, V, W><<<grid, kWideThreads, wide_tot_bytes<W>(), st>>>(g);                 \
  } while (0)
    if (bn == 112) {
      if (transA) { if (vec) RQLP_WIDE(true, true, 112); else RQLP_WIDE(true, false, 112); }
      else        { if (vec) RQLP_WIDE(false, true, 112); else RQLP_WIDE(false, false, 112); }
    } else {
      if (transA) { if (vec) RQLP_WIDE(true, true, 128); else RQLP_WIDE(true, false, 128); }
      else        { if (vec) RQLP_WIDE(false, true, 128); else RQLP_WIDE(false, false, 128); }
    }
#undef RQLP_WIDE
    note_launch();
  } else if (big && big_bn(g.N, g.K) == 32) {
    dim3 grid((unsigned)cdiv(g.N, 32), (unsigned)cdiv(g.M, 128), (unsigned)splits);
    if (transA) gemm_f32_kernel<128, 32, 16, 8, 4, true><<<grid, 128, 0, st>>>(g);
    else        gemm_f32_kernel<128, 32, 16, 8, 4, false><<<grid, 128, 0, st>>>(g);
    note_launch();
  } else if (big) {
    dim3 grid((unsigned)cdiv(g.N, 64), (unsigned)cdiv(g.M, 128), (unsigned)splits);
    if (transA) gemm_f32_kernel<128, 64, 16, 8, 4, true><<<grid, 256, 0, st>>>(g);
    else        gemm_f32_kernel<128, 64, 16, 8, 4, false><<<grid, 256, 0, st>>>(g);
    note_launch();
  } else {
    dim3 grid((unsigned)cdiv(g.N, 32), (unsigned)cdiv(g.M, 32), (unsigned)splits);
    if (transA) gemm_f32_kernel<32, 32, 16, 4, 4, true><<<grid, 64, 0, st>>>(g);
    else        gemm_f32_kernel<32, 32, 16, 4, 4, false><<<grid, 64, 0, st>>>(g);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t gemm_f32_ex(bool transA, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc, int splits, float* part,
                        double* sumsq, const int* gate, int gate_mode, bool b_upper, cudaStream_t st,
                        bool lower_only) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (lower_only && (M != N || use_wide(M, N, K))) return cudaErrorInvalidValue;
  if (gate != nullptr && gate_mode == kGateCopy && (transA || K != N)) return cudaErrorInvalidValue;
  if (gate != nullptr && gate_mode == kGateCopy) splits = 1;
  GemmArgs g;
  g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
  g.sumsq = sumsq; g.gate = gate; g.gate_mode = gate_mode; g.b_upper = b_upper ? 1 : 0;
  g.lower_only = lower_only ? 1 : 0;
  if (splits <= 1 || part == nullptr) {
    g.C = C; g.ldc = ldc; g.c_slice = 0; g.kchunk = round_up(K > 0 ? K : 1, 16);
    return launch_gemm(transA, g, 1, st);
  }
  g.C = part; g.ldc = N; g.c_slice = M * N;
  g.kchunk = round_up(cdiv(K, splits), 16);
  int used = (int)cdiv(K, g.kchunk);
  cudaError_t e = launch_gemm(transA, g, used, st);
  if (e != cudaSuccess) return e;
  int64_t total = M * N;
  int blocks = (int)std::min<int64_t>(cdiv(total, 256), (int64_t)sm_count() * 8);
  splitk_reduce_kernel<<<blocks, 256, 0, st>>>(M, N, used, part, C, ldc, lower_only ? 1 : 0,
                                                 gate_mode == kGateSkip ? gate : nullptr);
  note_launch();
  return cudaGetLastError();
}

// Grouped configurations (BM, BN, BK, TM, TN; threads = (BM/TM) (BN/TN)).
namespace {
// Resident CTAs per SM of one configuration (queried once; a launch with
// total <= 0 only primes the query, so that no query runs under capture).
// persistent: a few CTAs per SM walk the tile list; otherwise one CTA per
// tile and the hardware scheduler balances them.
template <int BM, int BN, int TM, int TN>
cudaError_t launch_grouped_cfg(bool transA, bool persistent, const GroupGemm* jobs, const int* tile_start,
                               int count, int total, cudaStream_t st) {
  constexpr int NT = (BM / TM) * (BN / TN);
  static int per_sm[2] = {0, 0};
  int& occ = per_sm[transA ? 1 : 0];
  if (occ == 0) {
    cudaError_t e = transA ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                 &occ, gemm_grouped_kernel<BM, BN, 16, TM, TN, true>, NT, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                 &occ, gemm_grouped_kernel<BM, BN, 16, TM, TN, false>, NT, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  if (total <= 0 || count <= 0) return cudaSuccess;
  const int grid = persistent ? std::max(1, std::min(total, sm_count() * occ)) : total;
  if (transA) gemm_grouped_kernel<BM, BN, 16, TM, TN, true><<<grid, NT, 0, st>>>(jobs, tile_start, count);
  else        gemm_grouped_kernel<BM, BN, 16, TM, TN, false><<<grid, NT, 0, st>>>(jobs, tile_start, count);
  note_launch();
  return cudaGetLastError();
}
}  // namespace

void grouped_tile(int cfg, int* bm, int* bn) {
  static const int kBM[kGroupCfgs] = {128, 64, 128, 64, 32, 32};
  static const int kBN[kGroupCfgs] = {64, 64, 32, 32, 32, 64};
  *bm = kBM[cfg];
  *bn = kBN[cfg];
}

cudaError_t gemm_grouped_prepare() {
  sm_count();
  for (int cfg = 0; cfg < kGroupChoices; ++cfg)
    for (int t = 0; t < 2; ++t) {
      cudaError_t e = gemm_grouped(t == 1, cfg, nullptr, nullptr, 0, 0, nullptr);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

cudaError_t gemm_grouped(bool transA, int choice, const GroupGemm* jobs, const int* tile_start, int count,
                         int total_tiles, cudaStream_t st) {
  const int cfg = choice % kGroupCfgs;
  const bool persistent = choice < kGroupCfgs;
#define RQLP_GROUPED(BM, BN, TM, TN) \
  launch_grouped_cfg<BM, BN, TM, TN>(transA, persistent, jobs, tile_start, count, total_tiles, st)
  switch (cfg) {
    case 0: return RQLP_GROUPED(128, 64, 8, 4);
    case 1: return RQLP_GROUPED(64, 64, 4, 4);
    case 2: return RQLP_GROUPED(128, 32, 8, 4);
    case 3: return RQLP_GROUPED(64, 32, 4, 4);
    case 4: return RQLP_GROUPED(32, 32, 4, 4);
    case 5: return RQLP_GROUPED(32, 64, 4, 4);
    // 8 x 8 outputs per thread: four 128-bit shared loads per 64 FMAs
    default: return cudaErrorInvalidValue;
  }
#undef RQLP_GROUPED
}

}  // namespace rqlp
