// Grouped tensor-core passes for the batched form (BF16x3): the passes over
// every problem's A of one step of the chain (Y = A^T X or Z = A X) in one
// launch.
//
// Per problem the batch plan holds A's BF16 halves in the 64-column panel
// layout of the single-problem engine (written once by split_grouped_kernel),
// the halves of the pass's X operand (X_hi^T, X_lo^T, K-major, written before
// every pass by prep_grouped_kernel) and eight tensor maps in device memory
// (A for both orientations, X for K = m and K = n). A work unit is one
// 128-row tile of one problem's output over that problem's whole K; the host
// balances the units over the CTAs (longest first, onto the least loaded
// CTA), so no tile is split and no CTA waits for another. Inside a CTA the
// pipeline is the single-problem pass kernel's: one TMA warp, one MMA warp
// (tcgen05.mma, M = 128, N = the problem's round16(d), FP32 accumulators in
// two TMEM buffers, the correction products in an accumulator of their own,
// chains cut every K = 4096), four epilogue warps. Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace rqlp {
namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128;
constexpr int BK = 32;                            // K per stage: 64-byte rows, 64B swizzle (K-major)
constexpr uint32_t kABytes = BM * BK * 2;         // one BF16 part of an A tile (8 KB)
constexpr int kThreads = 192;
constexpr int kMaxStages = 8;
constexpr int kChunkKB = 4096 / BK;               // k-blocks per accumulation chain
constexpr long long kWaitLimit = 4000000000LL;    // cycles (~2 s)

__device__ void post_timeout(int* info) {
  if (info != nullptr && atomicCAS(info, 0, RQLP_ERR_TIMEOUT) == 0) info[1] = 0;
}

template <bool MN_A>
__global__ void __launch_bounds__(kThreads, 1)
tc_grouped_kernel(const TcGJob* __restrict__ jobs, const int2* __restrict__ units, const int* __restrict__ cta_start,
                  int stages, uint32_t stage_bytes, uint32_t xslot, int npad_max, uint32_t tmem_cols, int* info,
                  int stall, int exact) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* epi_ok = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ub = cta_start[blockIdx.x], ue = cta_start[blockIdx.x + 1];
  if (ub >= ue) return;   // no units (uniform over the CTA)

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 4 * 32);
    }
    tc::mbar_init(done, 1);
    tc::fence_barrier_init();
  }
  if (warp == 5) {
    tc::tmem_alloc(tmem_slot, tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // Stage layout: A_hi, A_lo[, A_lo2] (kABytes each), then X_hi, X_lo[, X_lo2]
  // (xslot each).
  const bool ex = exact != 0;
  const uint32_t xoff = (ex ? 3u : 2u) * kABytes;

  if (warp == 4 && lane == 0) {
    // ------------------------------------------------ TMA producer
    long long issued = 0;
    bool ok = true;
    for (int ui = ub; ui < ue && ok; ++ui) {
      const int2 un = units[ui];
      const TcGJob& j = jobs[un.x];
      const int t = un.y;
      const CUtensorMap* mah = static_cast<const CUtensorMap*>(j.mAhi);
      const CUtensorMap* mal = static_cast<const CUtensorMap*>(j.mAlo);
      const CUtensorMap* mxh = static_cast<const CUtensorMap*>(j.mXhi);
      const CUtensorMap* mxl = static_cast<const CUtensorMap*>(j.mXlo);
      const CUtensorMap* mal2 = static_cast<const CUtensorMap*>(j.mAlo2);
      const CUtensorMap* mxl2 = static_cast<const CUtensorMap*>(j.mXlo2);
      const int nx = ex ? 3 : ((*j.xlo_nonzero) ? 2 : 1);
      const uint32_t xb = (uint32_t)j.npad * BK * 2;
      for (int kb = 0; kb < j.kblocks; ++kb, ++issued) {
        const int stage = (int)(issued % S);
        const uint32_t par = (uint32_t)((issued / S) & 1);
        if (!tc::mbar_wait(&empty[stage], par ^ 1u, kWaitLimit)) { ok = false; break; }
        // Test hook: CTA 0 withholds its first stage; the MMA warp's wait on
        // it, this thread's later waits and the epilogue's run out and report.
        if (stall != 0 && blockIdx.x == 0 && issued == 0) continue;
        unsigned char* base = smem + (size_t)stage * stage_bytes;
        tc::mbar_expect_tx(&full[stage], xoff + (uint32_t)nx * xb);
        if (MN_A) {   // 32 rows (K) of panels 2t and 2t + 1 (M)
          tc::tma_load_3d(base, mah, &full[stage], 0, kb * BK, 2 * t);
          tc::tma_load_3d(base + kABytes, mal, &full[stage], 0, kb * BK, 2 * t);
          if (ex) tc::tma_load_3d(base + 2 * kABytes, mal2, &full[stage], 0, kb * BK, 2 * t);
        } else {      // 128 rows (M) x 32 columns (K) of panel kb / 2
          const int kx = (kb & 1) * BK, kp = kb >> 1;
          tc::tma_load_3d(base, mah, &full[stage], kx, t * BM, kp);
          tc::tma_load_3d(base + kABytes, mal, &full[stage], kx, t * BM, kp);
          if (ex) tc::tma_load_3d(base + 2 * kABytes, mal2, &full[stage], kx, t * BM, kp);
        }
        tc::tma_load_2d(base + xoff, mxh, &full[stage], kb * BK, 0);
        if (nx >= 2) tc::tma_load_2d(base + xoff + xslot, mxl, &full[stage], kb * BK, 0);
        if (nx == 3) tc::tma_load_2d(base + xoff + 2 * xslot, mxl2, &full[stage], kb * BK, 0);
      }
    }
    if (!ok) post_timeout(info);
    for (long long i = issued > S ? issued - S : 0; i < issued; ++i)
      if (!tc::mbar_wait(&full[i % S], (uint32_t)((i / S) & 1), kWaitLimit)) post_timeout(info);
  } else if (warp == 5 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    long long consumed = 0;
    int seg = 0;
    bool ok = true;
    for (int ui = ub; ui < ue && ok; ++ui) {
      const TcGJob& j = jobs[units[ui].x];
      const int nx = ex ? 3 : ((*j.xlo_nonzero) ? 2 : 1);
      for (int s0 = 0; s0 < j.kblocks && ok; s0 += kChunkKB) {
        const int s1 = min(j.kblocks, s0 + kChunkKB);
        const int ab = seg & 1;
        if (!tc::mbar_wait(&acce[ab], (uint32_t)(((seg >> 1) & 1) ^ 1), kWaitLimit)) { ok = false; break; }
        tc::tc_fence_after();
        // Buffer ab holds A_hi X_hi in its first npad_max columns and the
        // correction products (~2^-8 of it) in the next npad_max: summed into
        // one accumulator they would lose bits to its magnitude at every MMA.
        const uint32_t d_tmem = tmem_base + (uint32_t)(ab * 2 * npad_max);
        const uint32_t d_corr = d_tmem + (uint32_t)npad_max;
        for (int kb = s0; kb < s1; ++kb, ++consumed) {
          const int stage = (int)(consumed % S);
          if (!tc::mbar_wait(&full[stage], (uint32_t)((consumed / S) & 1), kWaitLimit)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t base = tc::smem_u32(smem + (size_t)stage * stage_bytes);
          const uint32_t ahi = base, alo = base + kABytes, alo2 = base + 2 * kABytes, xhi = base + xoff,
                         xlo = xhi + xslot, xlo2 = xlo + xslot;
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            uint64_t dah, dal, dal2;
            if (MN_A) {   // MN-major, 128B swizzle: 16 k-rows = two 1024-byte atoms
              dah = tc::smem_desc(ahi + ks * 2048, kABytes / 2, 1024, tc::kSwizzle128);
              dal = tc::smem_desc(alo + ks * 2048, kABytes / 2, 1024, tc::kSwizzle128);
              dal2 = tc::smem_desc(alo2 + ks * 2048, kABytes / 2, 1024, tc::kSwizzle128);
            } else {      // K-major, 64B swizzle: 16 k-columns = 32 bytes into the row
              dah = tc::smem_desc(ahi + ks * 32, 16, 512, tc::kSwizzle64);
              dal = tc::smem_desc(alo + ks * 32, 16, 512, tc::kSwizzle64);
              dal2 = tc::smem_desc(alo2 + ks * 32, 16, 512, tc::kSwizzle64);
            }
            const uint64_t dxh = tc::smem_desc(xhi + ks * 32, 16, 512, tc::kSwizzle64);
            const uint64_t dxl = tc::smem_desc(xlo + ks * 32, 16, 512, tc::kSwizzle64);
            const uint64_t dxl2 = tc::smem_desc(xlo2 + ks * 32, 16, 512, tc::kSwizzle64);
            const uint32_t acc = (kb > s0 || ks > 0) ? 1u : 0u;
            tc::mma_bf16(d_tmem, dah, dxh, j.idesc, acc);
            if (nx >= 2) {
              tc::mma_bf16(d_corr, dah, dxl, j.idesc, acc);
              tc::mma_bf16(d_corr, dal, dxh, j.idesc, 1u);
            } else {
              tc::mma_bf16(d_corr, dal, dxh, j.idesc, acc);
            }
            if (ex) {   // the products above 2^-24 of the three-part operands
              tc::mma_bf16(d_corr, dal2, dxh, j.idesc, 1u);
              tc::mma_bf16(d_corr, dah, dxl2, j.idesc, 1u);
              tc::mma_bf16(d_corr, dal, dxl, j.idesc, 1u);
            }
          }
          tc::mma_commit(&empty[stage]);
        }
        if (!ok) break;
        tc::mma_commit(&accf[ab]);
        ++seg;
      }
    }
    if (!ok) post_timeout(info);
    tc::mma_commit(done);   // no MMA in flight at teardown
    if (!tc::mbar_wait(done, 0, kWaitLimit)) post_timeout(info);
  } else if (warp < 4) {
    // ------------------------------------------------ epilogue: TMEM -> global
    const int row = warp * 32 + lane;
    int seg = 0;
    bool ok = true;
    for (int ui = ub; ui < ue && ok; ++ui) {
      const int2 un = units[ui];
      const TcGJob& j = jobs[un.x];
      const long long gm = (long long)un.y * BM + row;
      float* dst = j.out + gm * j.ldo;
      const int ncols = gm < j.M ? j.d : 0;
      const bool vec = j.vec_out != 0;   // out rows 16-byte aligned
      for (int s0 = 0; s0 < j.kblocks; s0 += kChunkKB) {
        const int ab = seg & 1;
        // One thread waits; the verdict is shared so the four warps stay in step.
        if (threadIdx.x == 0) *epi_ok = tc::mbar_wait(&accf[ab], (uint32_t)((seg >> 1) & 1), kWaitLimit) ? 1 : 0;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (*epi_ok == 0) {
          if (threadIdx.x == 0) post_timeout(info);
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * 2 * npad_max);
        const bool first = s0 == 0;
        for (int c0 = 0; c0 < j.npad; c0 += 16) {   // uniform over the warp (collective TMEM loads)
          float v[16], w[16];
          tc::tmem_ld16(taddr + (uint32_t)c0, v);
          tc::tmem_ld16(taddr + (uint32_t)(npad_max + c0), w);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += w[i];
          if (vec && c0 + 16 <= ncols) {
            float4* d4 = reinterpret_cast<float4*>(dst + c0);
            if (!first) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float4 o = d4[q];
                v[4 * q] += o.x; v[4 * q + 1] += o.y; v[4 * q + 2] += o.z; v[4 * q + 3] += o.w;
              }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c0 + i < ncols) dst[c0 + i] = first ? v[i] : dst[c0 + i] + v[i];
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&acce[ab]);
        ++seg;
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 5) tc::tmem_dealloc(tmem_base, tmem_cols);
}

// Block -> problem: the last b with start[b] <= blk (start has count + 1 entries).
__device__ __forceinline__ int problem_of(const int* __restrict__ start, int count, int blk) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kSplitGroups = 2048;   // 8-element groups per block (256 threads x 8)

// Every problem's A (m x n FP32) -> A_hi, A_lo in 64-column panels (columns
// n..64 npan - 1 zero) and ||A||_F^2 (added to the problem's scalar).
__global__ void __launch_bounds__(256)
split_grouped_kernel(const SplitJob* __restrict__ jobs, const int* __restrict__ start, int count) {
  const int b = problem_of(start, count, blockIdx.x);
  const SplitJob j = jobs[b];
  const long long cpr = j.npan * 8, total = j.m * cpr;
  const long long g0 = (long long)(blockIdx.x - start[b]) * kSplitGroups;
  const bool vec = j.vec != 0;
  bf16* hi = reinterpret_cast<bf16*>(j.hi);
  bf16* lo = reinterpret_cast<bf16*>(j.lo);
  bf16* lo2 = reinterpret_cast<bf16*>(j.lo2);
  float s = 0.f, comp = 0.f;
  for (int it = 0; it < kSplitGroups / 256; ++it) {
    const long long g = g0 + it * 256 + threadIdx.x;
    if (g >= total) break;
    const long long r = g / cpr, c0 = (g % cpr) * 8;
    const float* src = j.A + r * j.lda + c0;
    float x[8];
    if (vec && c0 + 8 <= j.n) {
      const float4 p = *reinterpret_cast<const float4*>(src);
      const float4 q = *reinterpret_cast<const float4*>(src + 4);
      x[0] = p.x; x[1] = p.y; x[2] = p.z; x[3] = p.w; x[4] = q.x; x[5] = q.y; x[6] = q.z; x[7] = q.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = (c0 + i < j.n) ? src[i] : 0.f;
    }
    __align__(16) bf16 h[8];
    __align__(16) bf16 l[8];
    __align__(16) bf16 l2[8];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __float2bfloat16_rn(x[i]);
      const float r1 = x[i] - __bfloat162float(h[i]);   // exact in FP32
      l[i] = __float2bfloat16_rn(r1);
      l2[i] = __float2bfloat16_rn(r1 - __bfloat162float(l[i]));
      ss = fmaf(x[i], x[i], ss);
    }
    const long long o = ((c0 >> 6) * j.m + r) * 64 + (c0 & 63);
    *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(l);
    if (lo2 != nullptr) *reinterpret_cast<uint4*>(lo2 + o) = *reinterpret_cast<const uint4*>(l2);
    const float y = ss - comp, tt = s + y;
    comp = (tt - s) - y;
    s = tt;
  }
  __shared__ double red[8];
  double v = (double)s - (double)comp;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0 && j.sumsq != nullptr) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(j.sumsq, t);
  }
}

// Every problem's X (K x d FP32) -> X_hi^T, X_lo^T (d x ldk BF16, K-major);
// the problem's flag is raised when the low part is nonzero. One block per
// 64 (K) x 32 (d) tile, transposed through shared memory: tiles of problem b
// are numbered from start[b], row tiles fastest. Each thread writes two
// consecutive K entries of a column as one 32-bit pair (ldk is a multiple of
// 8, so a warp stores 128 contiguous bytes of a row of X^T); rows past K are
// read as zeros by the TMA.
constexpr int kPrepRows = 64;
__global__ void __launch_bounds__(256)
prep_grouped_kernel(const PrepJob* __restrict__ jobs, const int* __restrict__ start, int count) {
  __shared__ float tile[kPrepRows][33];
  const int b = problem_of(start, count, blockIdx.x);
  const PrepJob j = jobs[b];
  const int local = blockIdx.x - start[b];
  const int rtiles = (int)((j.K + kPrepRows - 1) / kPrepRows);
  const long long r0 = (long long)(local % rtiles) * kPrepRows;
  const int c0 = (local / rtiles) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < kPrepRows; i += 8) {
    const long long r = r0 + i;
    const int c = c0 + tx;
    tile[i][tx] = (r < j.K && c < j.d) ? j.X[r * j.ldx + c] : 0.f;
  }
  __syncthreads();
  bool any = false;
  bf16* th = reinterpret_cast<bf16*>(j.th);
  bf16* tl = reinterpret_cast<bf16*>(j.tl);
  bf16* tl2 = reinterpret_cast<bf16*>(j.tl2);
  const long long r = r0 + 2 * tx;   // this thread's pair of K entries (r + 1 < ldk when r < K)
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i;
    if (c >= j.d || r >= j.K) continue;
    bf16 h[2], l[2], l2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float x = tile[2 * tx + e][i];
      h[e] = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(h[e]);
      l[e] = __float2bfloat16_rn(r1);
      l2[e] = __float2bfloat16_rn(r1 - __bfloat162float(l[e]));
      any |= __bfloat162float(l[e]) != 0.f;
    }
    const long long o = (long long)c * j.ldk + r;
    *reinterpret_cast<__nv_bfloat162*>(th + o) = __halves2bfloat162(h[0], h[1]);
    *reinterpret_cast<__nv_bfloat162*>(tl + o) = __halves2bfloat162(l[0], l[1]);
    if (tl2 != nullptr) *reinterpret_cast<__nv_bfloat162*>(tl2 + o) = __halves2bfloat162(l2[0], l2[1]);
  }
  if (__syncthreads_or(any) && threadIdx.x == 0 && *(volatile int*)j.flag == 0) atomicOr(j.flag, 1);
}

size_t smem_optin() {
  static size_t v = 0;
  if (v == 0) {
    int dev = 0, x = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && x > 0)
      v = (size_t)x;
    else
      v = 227 * 1024;
  }
  return v;
}

template <bool MN_A>
cudaError_t launch_grouped(const TcGJob* jobs, const int2* units, const int* cta_start, int G, int npad_max,
                           int* info, int stall, bool exact, cudaStream_t st) {
  const uint32_t xslot = (uint32_t)npad_max * BK * 2;
  const uint32_t parts = exact ? 3u : 2u;
  const uint32_t stage_bytes = parts * kABytes + parts * xslot;
  const size_t avail = smem_optin() - 1024 - 512;
  const int S = std::max(1, std::min(kMaxStages, (int)(avail / stage_bytes)));
  // two buffers of (main, correction) accumulators: 4 npad_max <= 512 columns (d <= 128)
  if (4 * npad_max > 512) return cudaErrorInvalidValue;
  uint32_t tmem_cols = 32;
  while (tmem_cols < 4u * (uint32_t)npad_max) tmem_cols <<= 1;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc_grouped_kernel<MN_A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_optin());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (G <= 0) return cudaSuccess;   // configuration only
  const size_t smem = (size_t)S * stage_bytes + 1024 + 512;
  tc_grouped_kernel<MN_A><<<G, kThreads, smem, st>>>(jobs, units, cta_start, S, stage_bytes, xslot, npad_max,
                                                     tmem_cols, info, stall, exact ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host: tensor maps
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// BF16 tensor map of `rank` dims (innermost first), byte strides of dims 1.., box.
bool encode(void* map, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box, bool sw128) {
  EncodeFn fn = encoder();
  if (fn == nullptr) return false;
  cuuint32_t es[3] = {1, 1, 1};
  return fn(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank,
            const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            sw128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

static_assert(sizeof(CUtensorMap) == kTcMapBytes, "tensor map size");

bool tc_panel_map(void* map, const void* base, long long m, long long panels, int bi, int bo, int bp, bool sw128) {
  const cuuint64_t dims[3] = {64, (cuuint64_t)m, (cuuint64_t)panels};
  const cuuint64_t strides[2] = {128, (cuuint64_t)(m * 128)};
  const cuuint32_t box[3] = {(cuuint32_t)bi, (cuuint32_t)bo, (cuuint32_t)bp};
  return encode(map, base, 3, dims, strides, box, sw128);
}

bool tc_map2d(void* map, const void* base, long long inner, long long outer, long long pitch, int bi, int bo,
              bool sw128) {
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)bi, (cuuint32_t)bo};
  return encode(map, base, 2, dims, strides, box, sw128);
}

int tc_npad(int d) { return (int)round_up(std::max(d, 16), 16); }
uint32_t tc_idesc(int npad, bool a_mn_major) { return tc::idesc_bf16(BM, npad, a_mn_major, false); }

int tc_split_blocks(long long m, long long n) { return (int)cdiv(m * cdiv(n, 64) * 8, kSplitGroups); }
int tc_prep_blocks(long long K, int d) { return (int)(cdiv(K, kPrepRows) * cdiv(d, 32)); }

cudaError_t split_grouped(const SplitJob* jobs, const int* start, int count, int total_blocks, cudaStream_t st) {
  if (count <= 0 || total_blocks <= 0) return cudaSuccess;
  split_grouped_kernel<<<total_blocks, 256, 0, st>>>(jobs, start, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t prep_grouped(const PrepJob* jobs, const int* start, int count, int total_blocks, cudaStream_t st) {
  if (count <= 0 || total_blocks <= 0) return cudaSuccess;
  prep_grouped_kernel<<<total_blocks, 256, 0, st>>>(jobs, start, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t tc_grouped_pass(bool transA, const TcGJob* jobs, const int2* units, const int* cta_start, int G,
                            int npad_max, int* info, int stall, bool exact, cudaStream_t st) {
  return transA ? launch_grouped<true>(jobs, units, cta_start, G, npad_max, info, stall, exact, st)
                : launch_grouped<false>(jobs, units, cta_start, G, npad_max, info, stall, exact, st);
}

}  // namespace rqlp
