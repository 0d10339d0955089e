// Tensor-core passes over A in BF16 split precision (tcgen05 / TMEM / TMA).
//
// Each pass computes out = op(A) X with op(A) = A^T (Y = A^T X, the sketch
// and the A^T-half of a power pass) or A (Z = A X, the projection). A and X
// are split into BF16 high and low parts, A = A_hi + A_lo, X = X_hi + X_lo,
// and the product is accumulated in FP32 in tensor memory as
//     A_hi X_hi + A_hi X_lo + A_lo X_hi
// (the dropped A_lo X_lo term is below 2^-16 relative). When X has no low
// part (a BF16-exact Omega) the middle product is skipped.
//
// Exact mode (the products X R^{-1} of CholeskyQR, K = d): A and X in three
// parts each, A = A_hi + A_lo + A_lo2 (error 2^-27), and every product above
// 2^-27, A_hi X_hi + A_hi X_lo + A_lo X_hi + A_lo2 X_hi + A_hi X_lo2 +
// A_lo X_lo (six). R^{-1} spreads its entries over orders of magnitude, so
// the two-part form's error, relative to |X| |R^{-1}|, would be kappa(X)
// times larger relative to the result.
//
// Data flow per factorisation: split_a_kernel writes A_hi, A_lo once (and
// ||A||_F^2) in 64-column panels: panel c / 64 holds rows 0..m-1 of those
// 64 columns, 128 bytes per row, so that each part of an A tile is one TMA
// box (A^T X: 32 rows of two panels; A X: 128 rows of one panel);
// prep_x_kernel writes X_hi^T, X_lo^T (d x K, K-major) before
// every pass; tc_pass_kernel streams A tiles through shared memory with TMA
// and issues tcgen05.mma from one thread. A tile whose K range is split over
// several CTAs (stream-K) is finished by the CTA that arrives last on the
// tile's counter: it adds the published partial tiles in CTA order
// (deterministic) and resets the counter; no CTA ever waits for another.
//
// tc_pass_kernel is persistent: one CTA per SM, the (tile, k-block) units of
// the whole pass split evenly over the CTAs (stream-K), so the 157 M-tiles of
// a 20000-row pass load all 152 SMs equally. Warp roles: warps 0-3 drain the
// accumulator from TMEM (each warp its 32 lanes), warp 4 issues TMA loads,
// warp 5 allocates TMEM and issues the MMAs. Two accumulator buffers let the
// next segment's MMAs run while the epilogue drains the previous one. Every
// wait is bounded; a timeout is reported in the status word and the kernel
// drains what it started and frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace rqlp {
namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128;              // MMA M: output rows per tile (TMEM lanes)
constexpr int BK = 32;               // K per pipeline stage of the Gram kernel (64 bytes of BF16)
constexpr int kThreads = 192;        // 6 warps
constexpr int kMaxStages = 8;
constexpr long long kWaitLimit = 4000000000LL;   // cycles (~2 s) before a wait gives up
// K per pipeline stage of a pass: 64 (128-byte rows, 128B swizzle) where at
// least three such stages fit in shared memory, else 32 (64-byte rows, 64B
// swizzle). Larger TMA boxes stream A faster (measured: 7.1 vs 5.2 TB/s of
// A_hi + A_lo in the A^T X order at d = 64), but the pipeline needs stages in
// flight: at d = 224 only two K = 64 stages fit, and K = 32 with five is as fast.
constexpr int kMaxSlots = 16;                    // partial tiles summed from a cached slot list
// The FP32 accumulation of tcgen05.mma in TMEM loses a little of every add in
// the same direction: over K = 20000 a pass shrinks by ~1.5e-6 relative to
// its partial sums, which the cancelling small-singular-value columns of
// A P~ turn into ~1e-4 of their own size (and into the leading diagonal of
// L). Accumulation chains in TMEM are therefore cut every kChunkK of K
// (K = 4096); the epilogue adds the chunks in FP32 with round-to-nearest.
// The error falls linearly with the chunk (leading diagonal of L on the
// 20000^2 class: 4.2e-5, 2.1e-5, 9.4e-6 at K = 8192, 4096, 2048) and the time
// rises ~3% per halving.
constexpr int kChunkK = 4096;

struct TcArgs {
  int M, K, d, npad, kblocks, tiles, G, stages;
  int k0;                    // A^T X over A's rows k0 .. k0 + K - 1 (X holds those rows); 0 otherwise
  int m0;                    // A X over A's rows m0 .. m0 + M - 1 (out row 0 = A's row m0); 0 otherwise
  int tpc;                   // > 0: whole tiles per CTA (no split tiles); 0: stream-K
  int vec_out;               // out rows are 16-byte aligned (float4 stores)
  long long units;
  float* out;
  long long ldo;
  float* part;               // 2 * G slots of BM x npad floats
  int* tile_cnt;             // per-tile arrival counters (zero between passes)
  const int* xlo_nonzero;    // 1 when X has a nonzero low part
  int exact;                 // 1: A and X in three parts, six products
  int chunk;                 // k-blocks per accumulation chain in TMEM
  int split_acc;             // 1: correction products in their own accumulator
  int nbuf;                  // accumulator buffers (2: the epilogue overlaps the next chain)
  int bufcols;               // TMEM columns of one buffer (npad, or 2 npad when split_acc)
  int* info;                 // status word (may be null)
  uint32_t idesc, stage_bytes, tmem_cols;
  int fixup;                 // 1: split tiles are summed by tc_fixup_kernel after the pass
};

__host__ __device__ inline long long unit_begin(int c, long long units, int G) {
  return (long long)c * units / G;
}
// First unit of CTA c: stream-K (even split of all units) or, with tpc > 0,
// whole tiles (tpc tiles of kblocks units each per CTA).
__device__ inline long long cta_begin(const int c, const long long units, const int G, const int tpc,
                                      const int tiles, const int kblocks) {
  if (tpc > 0) return (long long)min(c * tpc, tiles) * kblocks;
  return unit_begin(c, units, G);
}
// The CTA whose unit range holds unit u (empty ranges never match).
__host__ __device__ inline int unit_owner(long long u, long long units, int G) {
  return (int)(((u + 1) * G + units - 1) / units) - 1;
}

// End of the accumulation chunk that starts at unit u (a CTA's range [.., u1)).
__device__ inline long long chunk_end(long long u, long long u1, int KB, int chunk) {
  const long long t_end = (u / KB + 1) * (long long)KB;
  return min(min(u1, t_end), u + chunk);
}

__device__ void post_timeout(int* info) {
  if (info != nullptr && atomicCAS(info, 0, RQLP_ERR_TIMEOUT) == 0) info[1] = 0;
}

template <bool MN_A, int BKP>
__global__ void __launch_bounds__(kThreads, 1)
tc_pass_kernel(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
               const __grid_constant__ CUtensorMap tmXhi, const __grid_constant__ CUtensorMap tmXlo,
               const __grid_constant__ CUtensorMap tmAlo2, const __grid_constant__ CUtensorMap tmXlo2,
               const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * a.stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* last_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* last_lo = last_flag + 1;
  int* epi_ok = last_lo + 2;
  int* nslots = epi_ok + 1;
  int* slots = nslots + 1;   // kMaxSlots entries

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cta = blockIdx.x;
  const long long u0 = cta_begin(cta, a.units, a.G, a.tpc, a.tiles, a.kblocks);
  const long long u1 = cta_begin(cta + 1, a.units, a.G, a.tpc, a.tiles, a.kblocks);
  if (u0 >= u1) return;   // no work for this CTA (uniform)
  const int KB = a.kblocks;

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
    tc::tmem_alloc(tmem_slot, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // Stage layout: A_hi, A_lo[, A_lo2], X_hi[, X_lo[, X_lo2]].
  const bool ex = a.exact != 0;
  const int nx = ex ? 3 : ((*a.xlo_nonzero) ? 2 : 1);
  constexpr uint32_t kAP = BM * BKP * 2;   // one BF16 A tile
  const int kChunk = a.chunk;
  constexpr uint32_t kRow = BKP * 2;        // bytes of a K-major row: the swizzle span
  constexpr uint32_t kSbo = 8 * kRow;       // 8-row swizzle atom of the K-major operands
  constexpr uint32_t kSw = BKP == 64 ? tc::kSwizzle128 : tc::kSwizzle64;
  const uint32_t xbytes = (uint32_t)a.npad * BKP * 2;
  const uint32_t xoff = (ex ? 3u : 2u) * kAP;

  if (warp == 4 && lane == 0) {
    // ------------------------------------------------ TMA producer
    tc::prefetch_tmap(&tmAhi);
    tc::prefetch_tmap(&tmAlo);
    tc::prefetch_tmap(&tmXhi);
    tc::prefetch_tmap(&tmXlo);
    if (ex) {
      tc::prefetch_tmap(&tmAlo2);
      tc::prefetch_tmap(&tmXlo2);
    }
    long long issued = 0;
    bool ok = true;
    for (long long u = u0; u < u1; ++u, ++issued) {
      const int stage = (int)(issued % S);
      const uint32_t par = (uint32_t)((issued / S) & 1);
      if (!tc::mbar_wait(&empty[stage], par ^ 1u, kWaitLimit)) { ok = false; break; }
      const int t = (int)(u / KB), kb = (int)(u % KB);
      unsigned char* base = smem + (size_t)stage * a.stage_bytes;
      tc::mbar_expect_tx(&full[stage], xoff + (uint32_t)nx * xbytes);
      // A maps are 3-D over the panel layout: {column in panel, row, panel}.
      if (MN_A) {   // 64 rows (K) of panels 2t and 2t + 1 (M), one box
        const int kr = a.k0 + kb * BKP;
        tc::tma_load_3d(base, &tmAhi, &full[stage], 0, kr, 2 * t);
        tc::tma_load_3d(base + kAP, &tmAlo, &full[stage], 0, kr, 2 * t);
        if (ex) tc::tma_load_3d(base + 2 * kAP, &tmAlo2, &full[stage], 0, kr, 2 * t);
      } else {      // 128 rows (M) x BKP columns (K) of panel kb BKP / 64
        const int kx = (kb * BKP) & 63, kp = (kb * BKP) >> 6, mr = a.m0 + t * BM;
        tc::tma_load_3d(base, &tmAhi, &full[stage], kx, mr, kp);
        tc::tma_load_3d(base + kAP, &tmAlo, &full[stage], kx, mr, kp);
        if (ex) tc::tma_load_3d(base + 2 * kAP, &tmAlo2, &full[stage], kx, mr, kp);
      }
      tc::tma_load_2d(base + xoff, &tmXhi, &full[stage], kb * BKP, 0);
      if (nx >= 2) tc::tma_load_2d(base + xoff + xbytes, &tmXlo, &full[stage], kb * BKP, 0);
      if (nx == 3) tc::tma_load_2d(base + xoff + 2 * xbytes, &tmXlo2, &full[stage], kb * BKP, 0);
    }
    if (!ok) post_timeout(a.info);
    // Drain: every load this thread started has landed before the CTA exits.
    for (long long i = issued > S ? issued - S : 0; i < issued; ++i)
      if (!tc::mbar_wait(&full[i % S], (uint32_t)((i / S) & 1), kWaitLimit)) post_timeout(a.info);
  } else if (warp == 5 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    long long consumed = 0;
    int seg = 0;
    bool ok = true;
    long long u = u0;
    while (u < u1 && ok) {
      const long long seg_begin = u, seg_end = chunk_end(u, u1, KB, kChunk);
      const int ab = seg % a.nbuf;
      if (!tc::mbar_wait(&acce[ab], (uint32_t)(((seg / a.nbuf) & 1) ^ 1), kWaitLimit)) { ok = false; break; }
      tc::tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(ab * a.bufcols);
      // The products of the low parts are ~2^-8 of A_hi X_hi or smaller. Added
      // into the same FP32 accumulator they lose bits to its large magnitude
      // at every MMA; with split_acc they accumulate on their own and the
      // epilogue adds the two sums with round-to-nearest.
      const uint32_t d_corr = a.split_acc ? d_tmem + (uint32_t)a.npad : d_tmem;
      for (; u < seg_end; ++u, ++consumed) {
        const int stage = (int)(consumed % S);
        if (!tc::mbar_wait(&full[stage], (uint32_t)((consumed / S) & 1), kWaitLimit)) { ok = false; break; }
        tc::tc_fence_after();
        const uint32_t base = tc::smem_u32(smem + (size_t)stage * a.stage_bytes);
        const uint32_t ahi = base, alo = base + kAP, alo2 = base + 2 * kAP, xhi = base + xoff,
                       xlo = xhi + xbytes, xlo2 = xlo + xbytes;
#pragma unroll
        for (int ks = 0; ks < BKP / 16; ++ks) {
          uint64_t dah, dal, dal2;
          if (MN_A) {   // MN-major, 128B swizzle: 16 k-rows = two 1024-byte atoms; panels kAP / 2 apart
            dah = tc::smem_desc(ahi + ks * 2048, kAP / 2, 1024, tc::kSwizzle128);
            dal = tc::smem_desc(alo + ks * 2048, kAP / 2, 1024, tc::kSwizzle128);
            dal2 = tc::smem_desc(alo2 + ks * 2048, kAP / 2, 1024, tc::kSwizzle128);
          } else {      // K-major: 16 k-columns = 32 bytes into the row
            dah = tc::smem_desc(ahi + ks * 32, 16, kSbo, kSw);
            dal = tc::smem_desc(alo + ks * 32, 16, kSbo, kSw);
            dal2 = tc::smem_desc(alo2 + ks * 32, 16, kSbo, kSw);
          }
          const uint64_t dxh = tc::smem_desc(xhi + ks * 32, 16, kSbo, kSw);
          const uint64_t dxl = tc::smem_desc(xlo + ks * 32, 16, kSbo, kSw);
          const uint64_t dxl2 = tc::smem_desc(xlo2 + ks * 32, 16, kSbo, kSw);
          const uint32_t acc = (u > seg_begin || ks > 0) ? 1u : 0u;
          // the first correction product of a chain starts d_corr when it is separate
          const uint32_t acc_c = a.split_acc ? acc : 1u;
          tc::mma_bf16(d_tmem, dah, dxh, a.idesc, acc);
          if (nx >= 2) {
            tc::mma_bf16(d_corr, dah, dxl, a.idesc, acc_c);
            tc::mma_bf16(d_corr, dal, dxh, a.idesc, 1u);
          } else {
            tc::mma_bf16(d_corr, dal, dxh, a.idesc, acc_c);
          }
          if (ex) {
            tc::mma_bf16(d_corr, dal2, dxh, a.idesc, 1u);
            tc::mma_bf16(d_corr, dah, dxl2, a.idesc, 1u);
            tc::mma_bf16(d_corr, dal, dxl, a.idesc, 1u);
          }
        }
        tc::mma_commit(&empty[stage]);
      }
      if (!ok) break;
      tc::mma_commit(&accf[ab]);
      ++seg;
    }
    if (!ok) post_timeout(a.info);
    tc::mma_commit(done);   // no MMA in flight at teardown
    if (!tc::mbar_wait(done, 0, kWaitLimit)) post_timeout(a.info);
  } else if (warp < 4) {
    // ------------------------------------------------ epilogue: TMEM -> global
    const int row = warp * 32 + lane;
    int seg = 0;
    long long u = u0;
    while (u < u1) {
      const int t = (int)(u / KB);
      const long long seg_begin = u, seg_end = chunk_end(u, u1, KB, kChunk);
      // This CTA's part of tile t, and where the chunk sits in it.
      const long long tb = std::max(u0, (long long)t * KB), te = std::min(u1, (long long)(t + 1) * KB);
      const bool whole = tb == (long long)t * KB && te == (long long)(t + 1) * KB;
      const bool first_chunk = seg_begin == tb, last_chunk = seg_end == te;
      const int ab = seg % a.nbuf;
      // One thread waits; the verdict is shared so the four warps stay in step.
      if (threadIdx.x == 0) *epi_ok = tc::mbar_wait(&accf[ab], (uint32_t)((seg / a.nbuf) & 1), kWaitLimit) ? 1 : 0;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (*epi_ok == 0) {
        if (threadIdx.x == 0) post_timeout(a.info);
        break;
      }
      tc::tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * a.bufcols);
      const long long gm = (long long)t * BM + row;
      float* dst;
      int ncols;
      if (whole) {
        dst = a.out + gm * a.ldo;
        ncols = gm < a.M ? a.d : 0;
      } else {
        const int slot = (tb == u0) ? 2 * cta : 2 * cta + 1;   // first or last tile of the range
        dst = a.part + ((long long)slot * BM + row) * a.npad;
        ncols = a.npad;
      }
      const bool vec = whole ? (a.vec_out != 0) : true;   // partial slots are 64-byte aligned
      // 32 columns per step: the row's earlier sums (this thread wrote them)
      // are all loaded before the step's stores, so the loads of a step
      // overlap instead of queueing behind stores to the same array.
      for (int c0 = 0; c0 < a.npad; c0 += 32) {
        float v[2][16];
        float4 o[2][4];
        float os[2][16];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = c0 + 16 * h;
          if (cc >= a.npad || first_chunk) continue;
          if (vec && cc + 16 <= ncols) {
            const float4* d4 = reinterpret_cast<const float4*>(dst + cc);
#pragma unroll
            for (int q = 0; q < 4; ++q) o[h][q] = d4[q];
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) os[h][i] = cc + i < ncols ? dst[cc + i] : 0.f;
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = c0 + 16 * h;
          if (cc >= a.npad) continue;   // uniform across the warp
          tc::tmem_ld16(taddr + (uint32_t)cc, v[h]);
          if (a.split_acc) {
            float w[16];
            tc::tmem_ld16(taddr + (uint32_t)(a.npad + cc), w);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[h][i] += w[i];
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = c0 + 16 * h;
          if (cc >= a.npad) continue;
          float* vv = v[h];
          if (vec && cc + 16 <= ncols) {
            float4* d4 = reinterpret_cast<float4*>(dst + cc);
            if (!first_chunk) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                vv[4 * q] += o[h][q].x; vv[4 * q + 1] += o[h][q].y;
                vv[4 * q + 2] += o[h][q].z; vv[4 * q + 3] += o[h][q].w;
              }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) d4[q] = make_float4(vv[4 * q], vv[4 * q + 1], vv[4 * q + 2], vv[4 * q + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (cc + i < ncols) dst[cc + i] = first_chunk ? vv[i] : os[h][i] + vv[i];
          }
        }
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&acce[ab]);
      if (!whole && last_chunk && !a.fixup) {
        // Publish the partial tile; the last CTA to arrive on the tile sums them.
        __threadfence();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (threadIdx.x == 0) {
          // Slots of this tile's contributors in CTA order (the fixed summation order).
          const long long ub = (long long)t * KB, ue = ub + KB;
          const int clo = unit_owner(ub, a.units, a.G), chi = unit_owner(ue - 1, a.units, a.G);
          int n = 0;
          for (int c = clo; c <= chi; ++c) {
            const long long cb = unit_begin(c, a.units, a.G);
            if (cb == unit_begin(c + 1, a.units, a.G)) continue;
            if (n < kMaxSlots) slots[n] = (cb / KB == t) ? 2 * c : 2 * c + 1;
            ++n;
          }
          const int old = atomicAdd(&a.tile_cnt[t], 1);
          *last_flag = (old == n - 1) ? 1 : 0;
          *nslots = n;
          last_lo[0] = clo;
          last_lo[1] = chi;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (*last_flag && *nslots <= kMaxSlots) {
          // Sum the slots in CTA order, the four warps over consecutive
          // float4 of the tile (coalesced), eight float4 per thread in flight.
          __threadfence();
          const int n = *nslots;
          const int Q = a.npad / 4, total = BM * Q;
          for (int f0 = threadIdx.x; f0 < total; f0 += 128 * 8) {
            float4 acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int s2 = 0; s2 < n; ++s2) {
              const float4* src = reinterpret_cast<const float4*>(a.part + (long long)slots[s2] * BM * a.npad);
              float4 v[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int f = f0 + 128 * j;
                v[j] = f < total ? __ldcg(src + f) : make_float4(0.f, 0.f, 0.f, 0.f);
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                acc[j].x += v[j].x; acc[j].y += v[j].y; acc[j].z += v[j].z; acc[j].w += v[j].w;
              }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int f = f0 + 128 * j;
              if (f >= total) continue;
              const int r = f / Q, c = (f % Q) * 4;
              const long long gr = (long long)t * BM + r;
              if (gr >= a.M || c >= a.d) continue;
              float* o = a.out + gr * a.ldo + c;
              if (a.vec_out && c + 3 < a.d) {
                *reinterpret_cast<float4*>(o) = acc[j];
              } else {
                const float w[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  if (c + i < a.d) o[i] = w[i];
              }
            }
          }
          if (threadIdx.x == 0) a.tile_cnt[t] = 0;
        } else if (*last_flag) {
          __threadfence();
          if (gm < a.M) {
            float* o = a.out + gm * a.ldo;
            for (int c0 = 0; c0 < a.d; c0 += 16) {
              float acc[16];
#pragma unroll
              for (int i = 0; i < 16; ++i) acc[i] = 0.f;
              {   // many contributors (tiny problems): recompute the slots
                for (int c = last_lo[0]; c <= last_lo[1]; ++c) {
                  const long long cb = unit_begin(c, a.units, a.G);
                  if (cb == unit_begin(c + 1, a.units, a.G)) continue;
                  const int slot = (cb / KB == t) ? 2 * c : 2 * c + 1;
                  const float4* src =
                      reinterpret_cast<const float4*>(a.part + ((long long)slot * BM + row) * a.npad + c0);
#pragma unroll
                  for (int q = 0; q < 4; ++q) {
                    const float4 v = __ldcg(src + q);
                    acc[4 * q] += v.x; acc[4 * q + 1] += v.y; acc[4 * q + 2] += v.z; acc[4 * q + 3] += v.w;
                  }
                }
              }
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (c0 + i < a.d) o[c0 + i] = acc[i];
            }
          }
          if (threadIdx.x == 0) a.tile_cnt[t] = 0;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      u = seg_end;
      ++seg;
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 5) tc::tmem_dealloc(tmem_base, a.tmem_cols);
}

// Sums of the split tiles when a tile has more contributors than the last
// arriver's slot list holds (few output tiles, e.g. A^T X with n <= ~1300):
// every split tile's partials are summed here by all SMs, one float4 of the
// output per thread, over the tile's contributors in CTA order (the order
// and the values of the last-arriver reduction).
__global__ void tc_fixup_kernel(const TcArgs a) {
  const int Q = a.npad / 4, KB = a.kblocks;
  const long long total = (long long)a.tiles * BM * Q;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(idx / ((long long)BM * Q));
    const int rem = (int)(idx % ((long long)BM * Q));
    const int r = rem / Q, c = (rem % Q) * 4;
    const long long gr = (long long)t * BM + r;
    if (gr >= a.M || c >= a.d) continue;
    const long long ub = (long long)t * KB, ue = ub + KB;
    const int clo = unit_owner(ub, a.units, a.G), chi = unit_owner(ue - 1, a.units, a.G);
    if (clo == chi) continue;   // one contributor: the tile was written whole
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int cc = clo; cc <= chi; ++cc) {
      const long long cb = unit_begin(cc, a.units, a.G);
      if (cb == unit_begin(cc + 1, a.units, a.G)) continue;
      const int slot = (cb / KB == t) ? 2 * cc : 2 * cc + 1;
      const float4 v = __ldcg(reinterpret_cast<const float4*>(a.part + ((long long)slot * BM + r) * a.npad + c));
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    float* o = a.out + gr * a.ldo + c;
    if (a.vec_out && c + 3 < a.d) {
      *reinterpret_cast<float4*>(o) = acc;
    } else {
      const float w[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (c + i < a.d) o[i] = w[i];
    }
  }
}

// Gram matrix of a split tall matrix on the tensor cores: G = X^T X for
// X = X_hi + X_lo (rows x cols, cols <= 256), products hi^T hi + hi^T lo +
// lo^T hi in FP32. CTA c takes an even share of the rows; each stage holds
// one 32-row chunk of X as 64-column MN-major boxes (128B swizzle), which
// serves as the A operand (X^T, one or two 128-row tiles of G, one TMEM
// accumulator each) and as the B operand (X, N = round16(cols)). Each CTA
// writes its partial G to its own slot; tc_gram_reduce_kernel adds the slots
// in CTA order.
struct GramArgs {
  int rows, cols, npad, kblocks, G, stages, mtiles, nbox;
  float* part;               // G slots of (mtiles * 128) x npad floats
  int* info;
  uint32_t idesc, stage_bytes, tmem_cols;
};

__global__ void __launch_bounds__(kThreads, 1)
tc_gram_kernel(const __grid_constant__ CUtensorMap tmHi, const __grid_constant__ CUtensorMap tmLo,
               const GramArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * a.stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* done = accf + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* epi_ok = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cta = blockIdx.x;
  const long long kb0 = unit_begin(cta, a.kblocks, a.G), kb1 = unit_begin(cta + 1, a.kblocks, a.G);
  const uint32_t half = (uint32_t)a.nbox * 4096u;   // bytes of one (hi or lo) chunk

  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < S; ++s2) {
      tc::mbar_init(&full[s2], 1);
      tc::mbar_init(&empty[s2], 1);
    }
    tc::mbar_init(accf, 1);
    tc::mbar_init(done, 1);
    tc::fence_barrier_init();
  }
  if (warp == 5) {
    tc::tmem_alloc(tmem_slot, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 4 && lane == 0) {
    tc::prefetch_tmap(&tmHi);
    tc::prefetch_tmap(&tmLo);
    long long issued = 0;
    bool ok = true;
    for (long long kb = kb0; kb < kb1; ++kb, ++issued) {
      const int stage = (int)(issued % S);
      if (!tc::mbar_wait(&empty[stage], (uint32_t)((issued / S) & 1) ^ 1u, kWaitLimit)) { ok = false; break; }
      unsigned char* base = smem + (size_t)stage * a.stage_bytes;
      tc::mbar_expect_tx(&full[stage], 2 * half);
      for (int b = 0; b < a.nbox; ++b) {   // panel b, 32 rows
        tc::tma_load_3d(base + b * 4096, &tmHi, &full[stage], 0, (int)(kb * BK), b);
        tc::tma_load_3d(base + half + b * 4096, &tmLo, &full[stage], 0, (int)(kb * BK), b);
      }
    }
    if (!ok) post_timeout(a.info);
    for (long long i = issued > S ? issued - S : 0; i < issued; ++i)
      if (!tc::mbar_wait(&full[i % S], (uint32_t)((i / S) & 1), kWaitLimit)) post_timeout(a.info);
  } else if (warp == 5 && lane == 0) {
    long long consumed = 0;
    bool ok = true;
    for (long long kb = kb0; kb < kb1; ++kb, ++consumed) {
      const int stage = (int)(consumed % S);
      if (!tc::mbar_wait(&full[stage], (uint32_t)((consumed / S) & 1), kWaitLimit)) { ok = false; break; }
      tc::tc_fence_after();
      const uint32_t hi = tc::smem_u32(smem + (size_t)stage * a.stage_bytes), lo = hi + half;
#pragma unroll
      for (int ks = 0; ks < BK / 16; ++ks) {
        const uint32_t koff = ks * 2048;
        const uint64_t bh = tc::smem_desc(hi + koff, 4096, 1024, tc::kSwizzle128);
        const uint64_t bl = tc::smem_desc(lo + koff, 4096, 1024, tc::kSwizzle128);
        for (int mt = 0; mt < a.mtiles; ++mt) {
          const uint64_t ah = tc::smem_desc(hi + mt * 8192 + koff, 4096, 1024, tc::kSwizzle128);
          const uint64_t al = tc::smem_desc(lo + mt * 8192 + koff, 4096, 1024, tc::kSwizzle128);
          const uint32_t d_tmem = tmem_base + (uint32_t)(mt * a.npad);
          const uint32_t acc = (kb > kb0 || ks > 0) ? 1u : 0u;
          tc::mma_bf16(d_tmem, ah, bh, a.idesc, acc);
          tc::mma_bf16(d_tmem, ah, bl, a.idesc, 1u);
          tc::mma_bf16(d_tmem, al, bh, a.idesc, 1u);
        }
      }
      tc::mma_commit(&empty[stage]);
    }
    if (!ok) post_timeout(a.info);
    tc::mma_commit(accf);
    tc::mma_commit(done);
    if (!tc::mbar_wait(done, 0, kWaitLimit)) post_timeout(a.info);
  } else if (warp < 4) {
    if (threadIdx.x == 0) *epi_ok = tc::mbar_wait(accf, 0, kWaitLimit) ? 1 : 0;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (*epi_ok == 0) {
      if (threadIdx.x == 0) post_timeout(a.info);
    } else {
      tc::tc_fence_after();
      const int row = warp * 32 + lane;
      for (int mt = 0; mt < a.mtiles; ++mt) {
        const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * a.npad);
        float* dst = a.part + ((long long)cta * a.mtiles * BM + mt * BM + row) * a.npad;
        for (int c0 = 0; c0 < a.npad; c0 += 16) {
          float v[16];
          tc::tmem_ld16(taddr + (uint32_t)c0, v);
          float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 5) tc::tmem_dealloc(tmem_base, a.tmem_cols);
}

// G[i][j] = sum over CTA slots of part (fixed order, Kahan-compensated FP32),
// for j <= i: the Cholesky reads the lower triangle only. Eight slots are
// loaded ahead of their adds, so a thread waits on about G / 8 round trips
// to L2 instead of G.
__global__ void tc_gram_reduce_kernel(const float* __restrict__ part, int G, int mtiles, int npad, int cols,
                                      float* __restrict__ out, long long ldo) {
  const long long slot = (long long)mtiles * BM * npad;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cols * cols; e += gridDim.x * blockDim.x) {
    const int i = e / cols, j = e % cols;
    if (j > i) continue;
    const float* p = part + (long long)i * npad + j;
    float s = 0.f, c = 0.f;
    int z = 0;
    for (; z + 8 <= G; z += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (long long)(z + u) * slot);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float y = v[u] - c, t = s + y;
        c = (t - s) - y;
        s = t;
      }
    }
    for (; z < G; ++z) {
      const float y = __ldcg(p + (long long)z * slot) - c, t = s + y;
      c = (t - s) - y;
      s = t;
    }
    out[(long long)i * ldo + j] = s;
  }
}

// A (m x n FP32) -> A_hi, A_lo (BF16) and ||A||_F^2, in 64-column panels:
// element (r, c) at ((c / 64) m + r) 64 + c % 64, columns n..npan*64-1 zero.
// lo2 (optional) receives bf16(A - A_hi - A_lo); both differences are exact in FP32.
// Rows row0 .. row0 + m - 1 of a matrix of mstride rows (the panel height).
__global__ void split_a_kernel(const float* __restrict__ A, long long m, long long n, long long lda, bool vec,
                               bf16* __restrict__ hi, bf16* __restrict__ lo, bf16* __restrict__ lo2, long long npan,
                               double* sumsq, long long mstride, long long row0) {
  const long long cpr = npan * 8, total = m * cpr;
  float s = 0.f, comp = 0.f;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / cpr, c0 = (idx % cpr) * 8;
    const float* src = A + r * lda + c0;
    float x[8];
    if (vec && c0 + 8 <= n) {
      const float4 p = *reinterpret_cast<const float4*>(src);
      const float4 q = *reinterpret_cast<const float4*>(src + 4);
      x[0] = p.x; x[1] = p.y; x[2] = p.z; x[3] = p.w; x[4] = q.x; x[5] = q.y; x[6] = q.z; x[7] = q.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = (c0 + i < n) ? src[i] : 0.f;
    }
    __align__(16) bf16 h[8];
    __align__(16) bf16 l[8];
    __align__(16) bf16 l2[8];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __float2bfloat16_rn(x[i]);
      const float r1 = x[i] - __bfloat162float(h[i]);
      l[i] = __float2bfloat16_rn(r1);
      l2[i] = __float2bfloat16_rn(r1 - __bfloat162float(l[i]));
      ss = fmaf(x[i], x[i], ss);
    }
    const long long o = ((c0 >> 6) * mstride + row0 + r) * 64 + (c0 & 63);
    *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(l);
    if (lo2 != nullptr) *reinterpret_cast<uint4*>(lo2 + o) = *reinterpret_cast<const uint4*>(l2);
    const float y = ss - comp, tt = s + y;
    comp = (tt - s) - y;
    s = tt;
  }
  if (sumsq == nullptr) return;
  __shared__ double red[32];
  double v = (double)s - (double)comp;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(sumsq, t);
  }
}

// X (rows x d FP32) -> X_hi^T, X_lo^T (d x ldk BF16, K-major); flags a nonzero low part.
// tl2 (optional) receives bf16(X - X_hi - X_lo). A block of 32 x 8 threads
// transposes a 64 (K) x 32 (d) tile through shared memory; each thread then
// writes two consecutive K entries of a column as one 32-bit pair, so a warp
// stores 128 contiguous bytes of a row of X^T (ldk is a multiple of 8).
constexpr int kPrepRows = 64;
__global__ void prep_x_kernel(const float* __restrict__ X, long long rows, int d, long long ldx,
                              bf16* __restrict__ th, bf16* __restrict__ tl, bf16* __restrict__ tl2, long long ldk,
                              int* nonzero_lo) {
  __shared__ float tile[kPrepRows][33];
  const long long r0 = (long long)blockIdx.x * kPrepRows;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < kPrepRows; i += blockDim.y) {
    const long long r = r0 + i;
    const int c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < d) ? X[r * ldx + c] : 0.f;
  }
  __syncthreads();
  bool any = false;
  const long long r = r0 + 2 * threadIdx.x;   // this thread's pair of K entries
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    if (c >= d || r >= ldk) continue;
    bf16 h[2], l[2], l2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float x = tile[2 * threadIdx.x + e][i];
      h[e] = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(h[e]);
      l[e] = __float2bfloat16_rn(r1);
      l2[e] = __float2bfloat16_rn(r1 - __bfloat162float(l[e]));
      any |= __bfloat162float(l[e]) != 0.f;
    }
    const long long o = (long long)c * ldk + r;
    *reinterpret_cast<__nv_bfloat162*>(th + o) = __halves2bfloat162(h[0], h[1]);
    *reinterpret_cast<__nv_bfloat162*>(tl + o) = __halves2bfloat162(l[0], l[1]);
    if (tl2 != nullptr) *reinterpret_cast<__nv_bfloat162*>(tl2 + o) = __halves2bfloat162(l2[0], l2[1]);
  }
  // One vote per block, and none once another block has raised the flag.
  if (__syncthreads_or(any) && threadIdx.x == 0 && threadIdx.y == 0 && *(volatile int*)nonzero_lo == 0)
    atomicOr(nonzero_lo, 1);
}

// ---------------------------------------------------------------- host side
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
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

// 2-D BF16 tensor map: dims {inner, outer}, row pitch in elements, box {bi, bo}.
bool make_map(CUtensorMap* map, const void* base, long long inner, long long outer, long long pitch, int bi,
              int bo, CUtensorMapSwizzle sw) {
  EncodeFn fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
  cuuint32_t box[2] = {(cuuint32_t)bi, (cuuint32_t)bo};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D BF16 tensor map over the 64-column panel layout of m rows: dims {64,
// m, panels}, box {bi, bo, bp}.
bool make_panel_map(CUtensorMap* map, const void* base, long long m, long long panels, int bi, int bo, int bp,
                    CUtensorMapSwizzle sw) {
  EncodeFn fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {64, (cuuint64_t)m, (cuuint64_t)panels};
  cuuint64_t strides[2] = {128, (cuuint64_t)(m * 128)};
  cuuint32_t box[3] = {(cuuint32_t)bi, (cuuint32_t)bo, (cuuint32_t)bp};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int npad_of(int d) { return (int)round_up(std::max(d, 16), 16); }
uint32_t tmem_cols_of(int cols) {
  uint32_t c = 32;
  while (c < (uint32_t)cols) c <<= 1;
  return c;
}
uint32_t stage_bytes_of(int npad, bool exact, int bkp) {
  return (exact ? 3u : 2u) * (uint32_t)(BM * bkp * 2) + (exact ? 3u : 2u) * (uint32_t)npad * bkp * 2;
}

size_t smem_optin_tc() {
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

// Pipeline stages of a pass (>= 1; the exact mode's stages at d = 256 hold
// one at a time, which its short K does not need more than).
int stages_of(int npad, bool exact, int bkp) {
  const size_t avail = smem_optin_tc() - 1024 - 512;
  int s = (int)(avail / stage_bytes_of(npad, exact, bkp));
  return std::max(1, std::min(kMaxStages, s));
}
int pass_bk(int npad, bool exact) { return stages_of(npad, exact, 64) >= 3 ? 64 : 32; }

template <bool MN_A, int BKP>
cudaError_t launch_pass(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& xh,
                        const CUtensorMap& xl, const CUtensorMap& al2, const CUtensorMap& xl2, const TcArgs& a,
                        cudaStream_t st) {
  const size_t smem = (size_t)a.stages * a.stage_bytes + 1024 + 512;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc_pass_kernel<MN_A, BKP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem_optin_tc()));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  tc_pass_kernel<MN_A, BKP><<<a.G, kThreads, smem, st>>>(ah, al, xh, xl, al2, xl2, a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(const float* A, int64_t lda, const float* Omega, int64_t ldo) {
  (void)A; (void)lda; (void)Omega; (void)ldo;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return false;
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

constexpr int kGramMaxCtas = 64;

void TcEngine::layout(Arena& ar, int64_t rows_cap, int64_t cols_cap, int d_cap, int64_t k_cap, bool gram,
                      bool three_part) {
  rows_cap_ = rows_cap;
  cols_cap_ = cols_cap;
  d_cap_ = d_cap;
  k_cap_ = k_cap;
  ldb_ = round_up(cols_cap, 64);   // whole 64-column panels
  G_ = sm_count();
  const int npad = npad_of(d_cap);
  Ahi_ = ar.take<uint16_t>((size_t)(rows_cap * ldb_));
  Alo_ = ar.take<uint16_t>((size_t)(rows_cap * ldb_));
  Alo2_ = three_part ? ar.take<uint16_t>((size_t)(rows_cap * ldb_)) : nullptr;
  Xhi_ = ar.take<uint16_t>((size_t)d_cap * round_up(k_cap, 8));
  Xlo_ = ar.take<uint16_t>((size_t)d_cap * round_up(k_cap, 8));
  Xlo2_ = three_part ? ar.take<uint16_t>((size_t)d_cap * round_up(k_cap, 8)) : nullptr;
  part_ = ar.take<float>((size_t)2 * G_ * BM * npad);
  flag_ = ar.take<int>(4);
  cnt_ = ar.take<int>((size_t)cdiv(std::max(rows_cap, cols_cap), BM));
  if (gram) {
    const int gp = npad_of((int)cols_cap);
    gpart_ = ar.take<float>((size_t)kGramMaxCtas * cdiv(cols_cap, BM) * BM * gp);
  }
}

cudaError_t TcEngine::split(const float* A, int64_t rows, int64_t cols, int64_t lda, double* sumsq,
                            cudaStream_t st) {
  if (rows > rows_cap_ || cols > cols_cap_) return cudaErrorInvalidValue;
  const bool vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda % 4 == 0);
  const long long npan = cdiv(cols, 64);
  const long long total = rows * npan * 8;
  const int blocks = (int)std::min<long long>(cdiv(total, 256), (long long)G_ * 8);
  split_a_kernel<<<blocks, 256, 0, st>>>(A, rows, cols, lda, vec, reinterpret_cast<bf16*>(Ahi_),
                                         reinterpret_cast<bf16*>(Alo_), reinterpret_cast<bf16*>(Alo2_), npan,
                                         sumsq, rows, 0);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  split_of_ = A;
  m_ = rows;
  n_ = cols;
  // Tile counters start at zero; each pass's last arrivals reset them.
  return cudaMemsetAsync(cnt_, 0, sizeof(int) * cdiv(std::max(rows_cap_, cols_cap_), BM), st);
}

cudaError_t TcEngine::begin_split(const float* A, int64_t rows, int64_t cols, cudaStream_t st) {
  if (rows > rows_cap_ || cols > cols_cap_) return cudaErrorInvalidValue;
  split_of_ = A;
  m_ = rows;
  n_ = cols;
  return cudaMemsetAsync(cnt_, 0, sizeof(int) * cdiv(std::max(rows_cap_, cols_cap_), BM), st);
}

cudaError_t TcEngine::split_rows(const float* Ablock, int64_t row0, int64_t rows, int64_t lda, double* sumsq,
                                 cudaStream_t st) {
  if (split_of_ == nullptr || row0 < 0 || row0 + rows > m_) return cudaErrorInvalidValue;
  const bool vec = (reinterpret_cast<uintptr_t>(Ablock) % 16 == 0) && (lda % 4 == 0);
  const long long npan = cdiv(n_, 64);
  const long long total = rows * npan * 8;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(cdiv(total, 256), (long long)G_ * 8));
  split_a_kernel<<<blocks, 256, 0, st>>>(Ablock, rows, n_, lda, vec, reinterpret_cast<bf16*>(Ahi_),
                                         reinterpret_cast<bf16*>(Alo_), reinterpret_cast<bf16*>(Alo2_), npan,
                                         sumsq, m_, row0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t TcEngine::pass(bool transA, const float* A, int64_t m, int64_t n, int64_t lda, const float* X,
                           int64_t ldx, int d, float* out, int64_t ldout, double* sumsq, int* info,
                           cudaStream_t st, bool exact) {
  if (split_of_ != A || m != m_ || n != n_) {
    cudaError_t e = split(A, m, n, lda, sumsq, st);
    if (e != cudaSuccess) return e;
  } else if (sumsq != nullptr) {
    return cudaErrorInvalidValue;   // ||A||^2 comes with the split only
  }
  return pass_k(transA, 0, transA ? m : n, X, ldx, d, out, ldout, info, st, exact);
}

cudaError_t TcEngine::pass_k(bool transA, int64_t k0, int64_t K, const float* X, int64_t ldx, int d, float* out,
                             int64_t ldout, int* info, cudaStream_t st, bool exact, int64_t m0, int64_t Mrows) {
  if (d > d_cap_ || split_of_ == nullptr) return cudaErrorInvalidValue;
  if (exact && (Alo2_ == nullptr || Xlo2_ == nullptr)) return cudaErrorInvalidValue;
  if (k0 < 0 || (!transA && k0 != 0) || k0 + K > (transA ? m_ : n_) || K <= 0) return cudaErrorInvalidValue;
  if (m0 < 0 || (transA && (m0 != 0 || Mrows >= 0)) || (!transA && Mrows >= 0 && m0 + Mrows > m_))
    return cudaErrorInvalidValue;
  cudaError_t e;
  const int64_t m = m_, n = n_;
  const int npad_ = npad_of(d);
  const long long M = transA ? n : (Mrows >= 0 ? Mrows : m);
  if (K > k_cap_) return cudaErrorInvalidValue;
  if ((e = cudaMemsetAsync(flag_, 0, sizeof(int), st)) != cudaSuccess) return e;
  {
    dim3 grid((unsigned)cdiv(round_up(K, 8), kPrepRows), (unsigned)cdiv(d, 32));
    prep_x_kernel<<<grid, dim3(32, 8), 0, st>>>(X, K, d, ldx, reinterpret_cast<bf16*>(Xhi_),
                                                 reinterpret_cast<bf16*>(Xlo_),
                                                 exact ? reinterpret_cast<bf16*>(Xlo2_) : nullptr, round_up(K, 8),
                                                 flag_);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  CUtensorMap ah, al, xh, xl, al2, xl2;
  const long long ldk = round_up(K, 8);
  bool ok;
  // The third parts are read in exact mode only; otherwise their maps repeat
  // the low parts'.
  const uint16_t* A3 = exact ? Alo2_ : Alo_;
  const uint16_t* X3 = exact ? Xlo2_ : Xlo_;
  const long long npan = cdiv(n, 64);
  const int bkp = pass_bk(npad_, exact);
  const CUtensorMapSwizzle ksw = bkp == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (transA) {   // op(A) = A^T: MN-major tiles, box 64 (j) x 32 (i) x 2 panels, 128B swizzle
    ok = make_panel_map(&ah, Ahi_, m, npan, 64, bkp, 2, CU_TENSOR_MAP_SWIZZLE_128B) &&
         make_panel_map(&al, Alo_, m, npan, 64, bkp, 2, CU_TENSOR_MAP_SWIZZLE_128B) &&
         make_panel_map(&al2, A3, m, npan, 64, bkp, 2, CU_TENSOR_MAP_SWIZZLE_128B);
  } else {        // op(A) = A: K-major tiles, box bkp (j) x 128 (i), swizzle = the row
    ok = make_panel_map(&ah, Ahi_, m, npan, bkp, BM, 1, ksw) &&
         make_panel_map(&al, Alo_, m, npan, bkp, BM, 1, ksw) &&
         make_panel_map(&al2, A3, m, npan, bkp, BM, 1, ksw);
  }
  ok = ok && make_map(&xh, Xhi_, K, d, ldk, bkp, npad_, ksw) &&
       make_map(&xl, Xlo_, K, d, ldk, bkp, npad_, ksw) &&
       make_map(&xl2, X3, K, d, ldk, bkp, npad_, ksw);
  if (!ok) return cudaErrorInvalidValue;

  TcArgs a;
  a.M = (int)M;
  a.K = (int)K;
  a.k0 = (int)k0;
  a.m0 = (int)m0;
  a.d = d;
  a.npad = npad_;
  a.kblocks = (int)cdiv(K, bkp);
  a.tiles = (int)cdiv(M, BM);
  a.units = (long long)a.tiles * a.kblocks;
  a.G = (int)std::min<long long>(G_, a.units);
  // Short K (e.g. X R^{-1} with K = d): split tiles would cost more in the
  // epilogue than they save, so give each CTA whole tiles.
  a.tpc = 0;
  if (a.kblocks <= 1024 / bkp) {
    a.tpc = (int)cdiv(a.tiles, G_);
    a.G = (int)cdiv(a.tiles, a.tpc);
  }
  // A tile spans at most G / tiles + 2 CTAs; past the last arriver's slot
  // list the split tiles are summed by tc_fixup_kernel instead.
  a.fixup = (a.tpc == 0 && (long long)a.G / a.tiles + 2 > kMaxSlots) ? 1 : 0;
  a.vec_out = ((reinterpret_cast<uintptr_t>(out) % 16) == 0 && ldout % 4 == 0) ? 1 : 0;
  a.exact = exact ? 1 : 0;
  a.chunk = kChunkK / bkp;
  // Correction products get their own accumulator where two such buffer
  // pairs fit in TMEM's 512 columns (npad <= 128), and always in exact mode
  // (single-buffered above npad = 128: the epilogue then holds the MMAs for
  // the drain of each chain).
  a.split_acc = (exact || 4 * npad_ <= 512) ? 1 : 0;
  a.bufcols = (a.split_acc ? 2 : 1) * npad_;
  a.nbuf = 2 * a.bufcols <= 512 ? 2 : 1;
  a.stages = stages_of(npad_, exact, bkp);
  a.out = out;
  a.ldo = ldout;
  a.part = part_;
  a.tile_cnt = cnt_;
  a.xlo_nonzero = flag_;
  a.info = info;
  a.idesc = tc::idesc_bf16(BM, npad_, transA, false);
  a.stage_bytes = stage_bytes_of(npad_, exact, bkp);
  a.tmem_cols = tmem_cols_of(a.nbuf * a.bufcols);
  const bool prof = profiled_ && profiling_on();
  if (prof) profile_mark_begin(st);
  if (bkp == 64)
    e = transA ? launch_pass<true, 64>(ah, al, xh, xl, al2, xl2, a, st)
               : launch_pass<false, 64>(ah, al, xh, xl, al2, xl2, a, st);
  else
    e = transA ? launch_pass<true, 32>(ah, al, xh, xl, al2, xl2, a, st)
               : launch_pass<false, 32>(ah, al, xh, xl, al2, xl2, a, st);
  if (e == cudaSuccess && a.fixup) {
    const long long total = (long long)a.tiles * BM * (npad_ / 4);
    const int blocks = (int)std::min<long long>(cdiv(total, 256), (long long)G_ * 8);
    tc_fixup_kernel<<<blocks, 256, 0, st>>>(a);
    note_launch();
    e = cudaGetLastError();
  }
  if (prof) profile_mark_end(st, transA ? 1 : 0);
  return e;
}

cudaError_t TcEngine::gram(float* Gout, int64_t ldg, int* info, cudaStream_t st) {
  if (split_of_ == nullptr || n_ > 256) return cudaErrorInvalidValue;
  const int cols = (int)n_;
  const int npad = npad_of(cols);
  const int mtiles = (int)cdiv(cols, BM);
  GramArgs a;
  a.rows = (int)m_;
  a.cols = cols;
  a.npad = npad;
  a.kblocks = (int)cdiv(m_, BK);
  a.G = std::max(1, std::min({a.kblocks / 8, kGramMaxCtas, G_}));
  a.mtiles = mtiles;
  a.nbox = std::max((int)cdiv(npad, 64), 2 * mtiles);
  a.stage_bytes = 2u * (uint32_t)a.nbox * 4096u;
  a.stages = std::max(2, std::min(kMaxStages, (int)((smem_optin_tc() - 1024 - 512) / a.stage_bytes)));
  a.part = gpart_;
  a.info = info;
  a.idesc = tc::idesc_bf16(BM, npad, true, true);
  {
    uint32_t need = (uint32_t)(mtiles * npad), c = 32;
    while (c < need) c <<= 1;
    a.tmem_cols = c;
  }
  CUtensorMap hi, lo;
  if (!make_panel_map(&hi, Ahi_, m_, cdiv(cols, 64), 64, BK, 1, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_panel_map(&lo, Alo_, m_, cdiv(cols, 64), 64, BK, 1, CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_optin_tc());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const size_t smem = (size_t)a.stages * a.stage_bytes + 1024 + 512;
  tc_gram_kernel<<<a.G, kThreads, smem, st>>>(hi, lo, a);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int blocks = std::max(1, std::min(G_ * 2, (cols * cols + 255) / 256));
  tc_gram_reduce_kernel<<<blocks, 256, 0, st>>>(gpart_, a.G, mtiles, npad, cols, Gout, ldg);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rqlp
