// Cholesky factor and inverse of the d x d Gram matrix of CholeskyQR, in one
// CTA: G = L L^T (R = L^T, upper, positive diagonal) and W = L^{-1}
// (R^{-1} = W^T).
//
// Blocked right-looking elimination on the augmented matrix [G | I] with
// 16-column panels J:
//   (1) warp 0 factors the 16 x 16 diagonal block L_JJ (row per lane,
//       right-looking, column t's entries broadcast by shuffles; each pivot
//       broadcast straight from its own lane's update);
//   (2) forward substitutions o = L_JJ^{-1} v, a thread per vector: the
//       panel L_IJ = G_IJ L_JJ^{-T} for the rows below, the block row of W
//       (W_J,: = L_JJ^{-1} X_J,:, X = the eliminated identity) and its
//       diagonal block L_JJ^{-1};
//   (3) trailing updates G_II -= L_IJ L_IJ^T (lower part) and
//       X_:J' -= L_IJ W_J,: for the rows above the next panel. The latter only
//       feeds later block rows of W, so it runs during the next panel's step
//       (1), on the warps that do not share warp 0's scheduler.
// Step (3) gives each warp 32 x 16 tiles and each lane 4 x 4 blocks, with the
// panel operands in transposed shared-memory buffers. L lives in the lower
// triangle of one square buffer and W^T in its strict upper triangle (W's
// diagonal in a side array). The Gram's lower triangle reaches shared memory
// by 16-byte asynchronous copies (FP32 factor, aligned rows), all of them in
// flight at once.
//
// A pivot that is not clearly positive restarts the elimination on G + s I
// (shifted CholeskyQR, Fukaya et al. 2020) and raises the caller's gate flag.
// The shift starts small, s0 = 10 d u trace(G), and grows tenfold while the
// shifted factor still breaks down (three shifts at most; then
// RQLP_ERR_BREAKDOWN and identities): X R^{-1} has condition number about
// sqrt(s / sigma_min(X)^2), so the smallest shift that factors leaves the
// least for the next CholeskyQR pass. With s0 = 100 d u trace(G) one FP32
// pass left a 317 x 66 sketch with kappa = 8e5 at kappa = 1.6e4, beyond what
// CholeskyQR2 can finish; with s0 = 10 d u trace(G), at 5e3.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rqlp {
namespace {

constexpr int NB = 16;
// Factorisation attempts: unshifted, then shifts s0, 10 s0, 100 s0 with
// s0 = 10 d u trace(G) (u: unit roundoff of the factor's type).
constexpr int kAttempts = 4;
constexpr int kMaxD = RQLP_MAX_D;
constexpr int kThreads = 512;
constexpr int kBatchThreads = 128;

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* v) {
  const typename Vec4<T>::type q = *reinterpret_cast<const typename Vec4<T>::type*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T* v) {
  typename Vec4<T>::type q;
  q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3];
  *reinterpret_cast<typename Vec4<T>::type*>(p) = q;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float u = 5.9604645e-8f; };
template <> struct Eps<double> { static constexpr double u = 1.1102230246251565e-16; };

// Row pitch of the square buffer: a multiple of 4 elements (16-byte rows) and
// 4 banks off a multiple of 32, so consecutive rows start in different banks.
__host__ __device__ inline int lds_of(int d) { return (int)round_up(d, 32) + 4; }
__host__ __device__ inline int ptld_of(int d) { return (int)round_up(d, 16); }

template <typename T> struct IsF32 { static constexpr bool value = false; };
template <> struct IsF32<float> { static constexpr bool value = true; };

__device__ void post_error(int* info, int code, int detail) {
  if (info != nullptr && atomicCAS(info, 0, code) == 0) info[1] = detail;
}

__device__ void write_identity(int d, float* R, float* Rinv, int64_t ldr) {
  for (int i = threadIdx.x >> 5; i < d; i += blockDim.x >> 5)
    for (int l = threadIdx.x & 31; l < d; l += 32) {
      const float v = i == l ? 1.f : 0.f;
      if (R != nullptr) R[i * ldr + l] = v;
      Rinv[i * ldr + l] = v;
    }
}

// Trailing update tiles of the panel that ends at column jn: lower: G_II -= L_IJ L_IJ^T over
// rows and columns [jn, d), c <= r (Ar = PT); else X -= L_IJ W_J,: over rows
// [0, jn), columns [jn, d) (Ar = WT). A warp takes a 32 x 16 tile (tiles w0,
// w0 + ws, ...), each lane a 4 x 4 block (lanes 8 x 4 over the tile): one k
// step reads 128 contiguous bytes of Ar and 64 of PT for the warp's 512
// FMAs, then a vectorised read-modify-write of S. Lower tiles: row strip q of
// 32 rows needs the column strips of 16 up to its diagonal (2 q + 2 of them).
template <typename T>
__device__ __forceinline__ void trailing_tiles(T* S, int LDS, const T* Ar, const T* PT, int d, int jn, bool lower,
                                               int w0, int ws, int lane) {
  const int PTLD = ptld_of(d), Nt = d - jn;
  if (Nt <= 0 || w0 < 0) return;
  const int nct = (Nt + 15) / 16;             // column strips over [jn, d)
  int ntiles = 0;
  if (lower) {
    const int nrs = (Nt + 31) / 32;           // row strips over [jn, d)
    for (int q = 0; q < nrs; ++q) ntiles += min(2 * q + 2, nct);
  } else {
    ntiles = ((jn + 31) / 32) * nct;
  }
  for (int t = w0; t < ntiles; t += ws) {
    int tr, tc, rlim;
    if (lower) {
      int q = 0, acc0 = 0;
      while (acc0 + min(2 * q + 2, nct) <= t) acc0 += min(2 * q++ + 2, nct);
      tr = jn + 32 * q;
      tc = jn + 16 * (t - acc0);
      rlim = d;
    } else {
      tr = 32 * (t / nct);
      tc = jn + 16 * (t % nct);
      rlim = jn;
    }
    const int r0 = tr + 4 * (lane >> 2), c0 = tc + 4 * (lane & 3);
    if (r0 < rlim && c0 < d && (!lower || c0 <= r0 + 3)) {
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        T av[4], bv[4];
        ld4(&Ar[k * PTLD + r0], av);
        ld4(&PT[k * PTLD + c0], bv);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + i;
        if (r >= rlim) continue;
        T sv[4];
        ld4(&S[(size_t)r * LDS + c0], sv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + j;
          if (c < d && (!lower || c <= r)) sv[j] -= acc[i][j];
        }
        st4(&S[(size_t)r * LDS + c0], sv);
      }
    }
  }
}

// The factorisation of one problem by the whole CTA (any multiple of 32
// threads up to kThreads). gS: the square buffer in global memory (used
// when !kShared).
template <typename T, bool kShared>
__device__ __forceinline__ void chol_body(int d, const float* __restrict__ G, int64_t ldg, float* __restrict__ R,
                                          float* __restrict__ Rinv, int64_t ldr, int* info, double* shift_count,
                                          int* gate_out, const int* gate_in, T* gS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LDS = lds_of(d), PTLD = ptld_of(d);
  T* dyn = reinterpret_cast<T*>(smem_raw);
  // kShared: S at the start of shared memory, so every access to it is a
  // shared-memory access; otherwise S = gS in global memory.
  T* S = kShared ? dyn : gS;
  T* PT = kShared ? dyn + (size_t)d * LDS : dyn;
  T* WT = PT + NB * PTLD;
  __shared__ __align__(32) T gdiag[kMaxD];
  __shared__ T wdiag[kMaxD];
  __shared__ T rdiag[NB];   // 1 / L_jj of the current diagonal block
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  if (gate_in != nullptr && *gate_in == 0) {   // pass not needed: R = R^{-1} = I
    write_identity(d, R, Rinv, ldr);
    return;
  }

  const T rel_tol = (T)64 * Eps<T>::u;
  T shift = 0;
  int fail = -1;
  for (int attempt = 0; attempt < kAttempts; ++attempt) {
    // attempt a >= 1 factors G + 10^(a-1) s0 I: the smallest shift that
    // succeeds reduces kappa(X R^{-1}) the most
    if (attempt > 1) shift *= (T)10;
    const T sh = attempt == 0 ? (T)0 : shift;
    // Lower triangle of G (+ sh I) into S, zeros above.
    bool loaded = false;
    if constexpr (kShared && IsF32<T>::value) {
      if ((reinterpret_cast<uintptr_t>(G) & 15) == 0 && (ldg & 3) == 0) {
        // 16-byte chunks: those that reach the diagonal are copied
        // asynchronously (all in flight at once), the others cleared; then
        // the diagonal chunk's entries above the diagonal are cleared and
        // the shift added. Chunk c of row i ends at 4 c + 3 < round_up(d, 4)
        // <= ldg, and S's rows hold LDS > 4 c + 3 entries.
        const int nch = (d + 3) >> 2;
        for (int e = tid; e < d * nch; e += blockDim.x) {
          const int i = e / nch, c4 = 4 * (e - i * nch);
          T* dst = &S[(size_t)i * LDS + c4];
          if (c4 <= i) {
            cp_async16(dst, &G[(int64_t)i * ldg + c4]);
          } else {
            const T z[4] = {(T)0, (T)0, (T)0, (T)0};
            st4(dst, z);
          }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int i = tid; i < d; i += blockDim.x) {
          const int ce = min(d, (i & ~3) + 4);
          for (int j = i + 1; j < ce; ++j) S[(size_t)i * LDS + j] = (T)0;
          const T x = S[(size_t)i * LDS + i] + sh;
          S[(size_t)i * LDS + i] = x;
          gdiag[i] = x;
        }
        loaded = true;
      }
    }
    // Otherwise a warp per group of four rows, lanes over columns, all of a
    // group's loads issued before its stores.
    for (int i0 = 4 * warp; !loaded && i0 < d; i0 += 4 * nwarps) {
      T v[4][kMaxD / 32];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < kMaxD / 32; ++t) {
          const int i = i0 + r, j = lane + 32 * t;
          v[r][t] = (i < d && j <= i) ? (T)G[(int64_t)i * ldg + j] : (T)0;
        }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < kMaxD / 32; ++t) {
          const int i = i0 + r, j = lane + 32 * t;
          if (i < d && j < d) {
            const T x = v[r][t] + (j == i ? sh : (T)0);
            S[(size_t)i * LDS + j] = x;
            if (j == i) gdiag[i] = x;
          }
        }
    }
    __syncthreads();
    if (attempt == 0) {   // trace(G), reduced by every warp in the same order
      T tr = 0;
      for (int i = lane; i < d; i += 32) tr += gdiag[i];
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      if (!isfinite(tr)) {
        if (tid == 0) post_error(info, RQLP_ERR_NONFINITE, 0);
        write_identity(d, R, Rinv, ldr);
        return;
      }
      shift = (T)(10.0 * d) * Eps<T>::u * tr;
    }
    fail = -1;
    // Panel loop. Phase B of panel J: warp 0 factors the diagonal block while
    // the other warps finish the previous panel's update of the rows above
    // (X -= L_IJ W_J,:, rows [0, j0)); the two touch disjoint parts of S.
    for (int j0 = 0; j0 < d; j0 += NB) {
      const int jb = min(NB, d - j0);
      const int jn = j0 + jb, Nt = d - jn;
      if (warp == 0) {
        // (1) L_JJ, lane = row, right-looking: column t is scaled by
        // 1 / sqrt(pivot), then every later column c takes l_it l_ct (l_ct
        // from lane c by a shuffle). Only column t + 1's update lies on the
        // path to the next pivot. Branch-free; entries above the diagonal are
        // cleared before the store.
        T l[NB], gd[NB];
#pragma unroll
        for (int k = 0; k < NB; k += 4) {
          if (lane < jb) ld4(&S[(size_t)(j0 + lane) * LDS + j0 + k], &l[k]);
          else l[k] = l[k + 1] = l[k + 2] = l[k + 3] = (T)0;
          ld4(&gdiag[j0 + k], &gd[k]);
        }
        int f = -1;
        T piv = __shfl_sync(0xffffffffu, l[0], 0);
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          const bool live = t < jb;
          const bool ok = piv > rel_tol * gd[t] && isfinite(piv);
          f = (f < 0 && live && !ok) ? j0 + t : f;
          const T rl = rsqrt(ok ? piv : (T)1);
          if (lane == 0) rdiag[t] = rl;
          l[t] = lane == t ? piv * rl : (lane > t ? l[t] * rl : (T)0);
          // The next pivot is lane t + 1's own update of its diagonal entry
          // (the operation the column loop below performs there, so the same
          // value), broadcast without waiting on the shuffle of column t.
          if (t + 1 < NB) piv = __shfl_sync(0xffffffffu, l[t + 1] - l[t] * l[t], t + 1);
#pragma unroll
          for (int c = t + 1; c < NB; ++c) l[c] -= l[t] * __shfl_sync(0xffffffffu, l[t], c);
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k > lane) l[k] = (T)0;
        if (f < 0 && lane < jb) {   // zeros above the diagonal: W's block there is written in (2)
#pragma unroll
          for (int k = 0; k < NB; k += 4) st4(&S[(size_t)(j0 + lane) * LDS + j0 + k], &l[k]);
        }
        if (lane == 0) s_fail = f;
      }
      // The update of the rows above goes to the warps that do not share warp
      // 0's scheduler (warp % 4 != 0), so that the serial factor issues alone.
      if (j0 > 0) {
        if (nwarps >= 8) {
          if ((warp & 3) != 0)
            trailing_tiles<T>(S, LDS, WT, PT, d, j0, false, (warp >> 2) * 3 + (warp & 3) - 1, (nwarps >> 2) * 3, lane);
        } else if (warp > 0 || nwarps == 1) {
          trailing_tiles<T>(S, LDS, WT, PT, d, j0, false, nwarps > 1 ? warp - 1 : 0, max(nwarps - 1, 1), lane);
        }
      }
      __syncthreads();
      if (s_fail >= 0) {
        fail = s_fail;
        break;
      }
      // (2) o = L_JJ^{-1} v by forward substitution, a thread per vector:
      // panel rows below (v = G_IJ row, o = L_IJ row -> S and PT), rows of
      // W's block row J (v = the eliminated identity's column, o -> S and
      // WT) and W's diagonal block (v = unit vector, o = column of D).
      for (int idx = tid; idx < Nt + jn; idx += blockDim.x) {
        T v[NB];
        int src = -1;   // row of S that holds v, or -1 for a unit vector
        if (idx < Nt) src = jn + idx;
        else if (idx - Nt < j0) src = idx - Nt;
        const int cc = idx - Nt - j0;   // diagonal-block column (unit vector e_cc)
        if (src >= 0) {
#pragma unroll
          for (int k = 0; k < NB; k += 4) ld4(&S[(size_t)src * LDS + j0 + k], &v[k]);
          if (jb < NB) {
#pragma unroll
            for (int k = 0; k < NB; ++k)
              if (k >= jb) v[k] = (T)0;
          }
        } else {
#pragma unroll
          for (int k = 0; k < NB; ++k) v[k] = k == cc ? (T)1 : (T)0;
        }
        T o[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < jb) {
            const T* lr = &S[(size_t)(j0 + c) * LDS + j0];
            T sacc = v[c];
#pragma unroll
            for (int k = 0; k < c; k += 4) {
              T lv[4];
              ld4(&lr[k], lv);
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (k + u < c) sacc -= lv[u] * o[k + u];
            }
            o[c] = sacc * rdiag[c];
          } else {
            o[c] = (T)0;
          }
        }
        if (idx < Nt) {
          const int i = jn + idx;
#pragma unroll
          for (int c = 0; c < NB; ++c) PT[c * PTLD + i] = o[c];
#pragma unroll
          for (int k = 0; k < NB; k += 4) st4(&S[(size_t)i * LDS + j0 + k], &o[k]);
        } else if (src >= 0) {
#pragma unroll
          for (int rr = 0; rr < NB; ++rr) {
            if (rr < jb) {
              S[(size_t)src * LDS + j0 + rr] = o[rr];
              WT[rr * PTLD + src] = o[rr];
            }
          }
        } else {
          const int c = j0 + cc;
          wdiag[c] = rdiag[cc];   // = o[cc]
#pragma unroll
          for (int rr = 0; rr < NB; ++rr) {
            if (rr < jb) {
              if (rr > cc) S[(size_t)c * LDS + j0 + rr] = o[rr];
              WT[rr * PTLD + c] = o[rr];
            }
          }
        }
      }
      __syncthreads();
      // (3) trailing update G_II -= L_IJ L_IJ^T of the lower part; the rows
      // above follow in the next panel's phase B.
      if (Nt > 0) trailing_tiles<T>(S, LDS, PT, PT, d, jn, true, warp, nwarps, lane);
      __syncthreads();
    }
    if (fail < 0) break;
    __syncthreads();
    if (attempt == 0 && tid == 0) {
      if (gate_out != nullptr) *gate_out = 1;
      if (shift_count != nullptr) atomicAdd(shift_count, 1.0);
    }
  }

  if (fail >= 0) {
    if (tid == 0) post_error(info, RQLP_ERR_BREAKDOWN, fail + 1);
    write_identity(d, R, Rinv, ldr);
    return;
  }
  // R = L^T (upper); R^{-1} = W^T: strict upper part from S, diagonal from wdiag.
  for (int i = warp; i < d; i += nwarps) {   // a warp per row, lanes over columns
    float* r = R != nullptr ? R + (int64_t)i * ldr : nullptr;
    float* ri = Rinv + (int64_t)i * ldr;
    for (int l = lane; l < d; l += 32) {
      if (R != nullptr) r[l] = l >= i ? (float)S[(size_t)l * LDS + i] : 0.f;
      ri[l] = l > i ? (float)S[(size_t)i * LDS + l] : (l == i ? (float)wdiag[i] : 0.f);
    }
  }
}

template <typename T, bool kShared>
__global__ void __launch_bounds__(kThreads)
chol_blocked_kernel(int d, const float* __restrict__ G, int64_t ldg, float* __restrict__ R, float* __restrict__ Rinv,
                    int64_t ldr, int* info, double* shift_count, int* gate_out, const int* gate_in, T* gS) {
  chol_body<T, kShared>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in, gS);
}

// One CTA per problem of a batch; every square buffer in shared memory.
template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 3)
chol_batched_kernel(const CholJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x;
  if (b >= count) return;
  const CholJob j = jobs[b];
  chol_body<T, true>(j.d, j.G, j.ldg, j.R, j.Rinv, j.ldr, j.info, j.shift_count, j.gate_out, j.gate_in, nullptr);
}

size_t smem_optin_chol() {
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

template <typename T>
size_t square_bytes(int d) { return (size_t)d * lds_of(d) * sizeof(T); }
template <typename T>
size_t panel_bytes(int d) { return (size_t)2 * NB * ptld_of(d) * sizeof(T); }
template <typename T>
size_t static_bytes() { return (2 * kMaxD + NB) * sizeof(T) + 96; }
template <typename T>
bool square_in_smem(int d) {
  return square_bytes<T>(d) + panel_bytes<T>(d) + static_bytes<T>() <= smem_optin_chol();
}

template <typename T>
cudaError_t launch(int d, const float* G, int64_t ldg, float* R, float* Rinv, int64_t ldr, int* info,
                   double* shift_count, int* gate_out, const int* gate_in, void* gstore, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    const int cap = (int)(smem_optin_chol() - static_bytes<T>());
    cudaError_t e = cudaFuncSetAttribute(chol_blocked_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(chol_blocked_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const bool in_smem = square_in_smem<T>(d);
  if (!in_smem && gstore == nullptr) return cudaErrorInvalidValue;
  const size_t dyn = panel_bytes<T>(d) + (in_smem ? square_bytes<T>(d) : 0);
  if (in_smem)
    chol_blocked_kernel<T, true><<<1, kThreads, dyn, st>>>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out,
                                                           gate_in, nullptr);
  else
    chol_blocked_kernel<T, false><<<1, kThreads, dyn, st>>>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out,
                                                            gate_in, reinterpret_cast<T*>(gstore));
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batched(const CholJob* jobs, int count, int dmax, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(chol_batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem_optin_chol() - static_bytes<T>()));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (count <= 0) return cudaSuccess;   // configuration only
  if (!square_in_smem<T>(dmax)) return cudaErrorInvalidValue;
  const size_t dyn = panel_bytes<T>(dmax) + square_bytes<T>(dmax);
  chol_batched_kernel<T><<<count, kBatchThreads, dyn, st>>>(jobs, count);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool chol_batched_fits(int dmax, bool fp64) {
  return fp64 ? square_in_smem<double>(dmax) : square_in_smem<float>(dmax);
}

cudaError_t chol_inv_batched(const CholJob* jobs, int count, int dmax, bool fp64, cudaStream_t st) {
  return fp64 ? launch_batched<double>(jobs, count, dmax, st) : launch_batched<float>(jobs, count, dmax, st);
}

size_t chol_global_bytes(int d, bool fp64) {
  if (fp64) return square_in_smem<double>(d) ? 0 : square_bytes<double>(d);
  return square_in_smem<float>(d) ? 0 : square_bytes<float>(d);
}

cudaError_t chol_inv(int d, const float* G, int64_t ldg, float* R, float* Rinv, int64_t ldr, int* info,
                     double* shift_count, int* gate_out, const int* gate_in, void* gstore, bool fp64,
                     cudaStream_t st) {
  if (fp64) return launch<double>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in, gstore, st);
  return launch<float>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in, gstore, st);
}

}  // namespace rqlp
