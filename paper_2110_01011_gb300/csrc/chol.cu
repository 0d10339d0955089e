// Cholesky factor and inverse of the d x d Gram matrix of CholeskyQR, in one
// CTA: G = L L^T (R = L^T, upper, positive diagonal) and W = L^{-1}
// (R^{-1} = W^T).
//
// Blocked right-looking elimination on the augmented matrix [G | I] with
// 16-column panels:
//   (1) one warp factors the 16 x 16 diagonal block (left-looking, row per
//       lane, rows of L_JJ broadcast by shuffles) and inverts it (column per
//       lane, same broadcasts): L_JJ, D = L_JJ^{-1};
//   (2) panel L_IJ = G_IJ D^T for the rows below, and the block row of W:
//       W_J,: = D X_J,: (X = the eliminated identity, W_JJ = D);
//   (3) trailing updates G_II -= L_IJ L_IJ^T (lower part) and
//       X_I,: -= L_IJ W_J,: for the rows below.
// Step (3) gives each thread 4 x 4 blocks of outputs, with the panel operands
// in transposed shared-memory buffers (one 128-bit load of row values and one
// of column values per 16 FMAs). L lives in the lower triangle of one square buffer and
// W^T in its strict upper triangle (W's diagonal in a side array).
//
// A pivot that is not clearly positive restarts the elimination on G + s I
// (shifted CholeskyQR, Fukaya et al. 2020) and raises the caller's gate flag;
// a second breakdown reports RQLP_ERR_BREAKDOWN and writes identities.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rqlp {
namespace {

constexpr int NB = 16;
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

__device__ void post_error(int* info, int code, int detail) {
  if (info != nullptr && atomicCAS(info, 0, code) == 0) info[1] = detail;
}

__device__ void write_identity(int d, float* R, float* Rinv, int64_t ldr) {
  for (int i = threadIdx.x >> 5; i < d; i += blockDim.x >> 5)
    for (int l = threadIdx.x & 31; l < d; l += 32) {
      const float v = i == l ? 1.f : 0.f;
      R[i * ldr + l] = v;
      Rinv[i * ldr + l] = v;
    }
}

// The factorisation of one problem by the whole CTA (any multiple of 32
// threads up to kThreads). gS: the square buffer in global memory, or nullptr
// for shared memory.
template <typename T>
__device__ __forceinline__ void chol_body(int d, const float* __restrict__ G, int64_t ldg, float* __restrict__ R,
                                          float* __restrict__ Rinv, int64_t ldr, int* info, double* shift_count,
                                          int* gate_out, const int* gate_in, T* gS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LDS = lds_of(d), PTLD = ptld_of(d);
  T* dyn = reinterpret_cast<T*>(smem_raw);
  T* S = gS != nullptr ? gS : dyn;
  T* PT = gS != nullptr ? dyn : dyn + (size_t)d * LDS;
  T* WT = PT + NB * PTLD;
  __shared__ T gdiag[kMaxD], wdiag[kMaxD];
  __shared__ __align__(32) T Dinv[NB][NB];   // D = L_JJ^{-1}, zero above the diagonal and beyond jb
  __shared__ T rdiag[NB];
  __shared__ T s_red[32];
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  if (gate_in != nullptr && *gate_in == 0) {   // pass not needed: R = R^{-1} = I
    write_identity(d, R, Rinv, ldr);
    return;
  }

  T tr = 0;
  for (int i = tid; i < d; i += blockDim.x) tr += (T)G[(int64_t)i * ldg + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
  if (lane == 0) s_red[warp] = tr;
  __syncthreads();
  T trace = 0;
  for (int w = 0; w < nwarps; ++w) trace += s_red[w];
  if (!isfinite(trace)) {
    if (tid == 0) post_error(info, RQLP_ERR_NONFINITE, 0);
    write_identity(d, R, Rinv, ldr);
    return;
  }
  const T shift = (T)(100.0 * d) * Eps<T>::u * trace;
  const T rel_tol = (T)64 * Eps<T>::u;

  int fail = -1;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const T sh = attempt == 0 ? (T)0 : shift;
    // Lower triangle of G (+ sh I) into S, zeros above: a warp per pair of
    // rows, lanes over columns, all of a pair's loads issued before its stores.
    for (int i0 = 2 * warp; i0 < d; i0 += 2 * nwarps) {
      T v[2][kMaxD / 32];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int t = 0; t < kMaxD / 32; ++t) {
          const int i = i0 + r, j = lane + 32 * t;
          v[r][t] = (i < d && j <= i) ? (T)G[(int64_t)i * ldg + j] : (T)0;
        }
#pragma unroll
      for (int r = 0; r < 2; ++r)
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
    fail = -1;
    for (int j0 = 0; j0 < d; j0 += NB) {
      const int jb = min(NB, d - j0);
      // (1) diagonal block, warp 0 (lane = row): left-looking Cholesky, row j
      // of L_JJ broadcast by shuffles, one reciprocal square root per column;
      // then D = L_JJ^{-1} with lane = column, rows of L_JJ broadcast the same
      // way. Everything stays in registers until the results are stored.
      if (warp == 0) {
        T l[NB];
#pragma unroll
        for (int k = 0; k < NB; k += 4) {
          if (lane < jb) ld4(&S[(size_t)(j0 + lane) * LDS + j0 + k], &l[k]);
          else l[k] = l[k + 1] = l[k + 2] = l[k + 3] = (T)0;
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k > lane) l[k] = (T)0;
        int f = -1;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          if (j < jb && f < 0) {
            T s = l[j];                       // a_ij - sum_{t<j} l_it l_jt
#pragma unroll
            for (int t = 0; t < j; ++t) s -= l[t] * __shfl_sync(0xffffffffu, l[t], j);
            const T piv = __shfl_sync(0xffffffffu, s, j);
            if (!(piv > rel_tol * gdiag[j0 + j]) || !isfinite(piv)) {
              f = j0 + j;
            } else {
              const T rl = rsqrt(piv);
              if (lane == 0) rdiag[j] = rl;
              l[j] = lane == j ? piv * rl : (lane > j ? s * rl : (T)0);
            }
          }
        }
        if (f < 0) {
#pragma unroll
          for (int k = 0; k < NB; ++k)
            if (lane < jb && k <= lane) S[(size_t)(j0 + lane) * LDS + j0 + k] = l[k];
          __syncwarp();
          const int c = lane;   // column of D: x[i] = D_ic
          T x[NB];
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            T s = 0;
#pragma unroll
            for (int t = 0; t < i; ++t) s += __shfl_sync(0xffffffffu, l[t], i) * x[t];
            const T ri = rdiag[i];
            x[i] = (i < c || i >= jb) ? (T)0 : (i == c ? ri : -s * ri);
          }
          if (c < NB) {
#pragma unroll
            for (int i = 0; i < NB; ++i) Dinv[i][c] = (c < jb && i < jb) ? x[i] : (T)0;
          }
        }
        if (lane == 0) s_fail = f;
      }
      __syncthreads();
      if (s_fail >= 0) {
        fail = s_fail;
        break;
      }
      const int jn = j0 + jb, Nt = d - jn;
      // (2) panel rows below the block, block row of W, and W's diagonal
      // block. Two threads per row, one for the even and one for the odd
      // outputs, each reading rows of D as 128-bit broadcasts; results are
      // computed in registers and stored afterwards.
      for (int task = tid; task < 2 * (Nt + jn); task += blockDim.x) {
        const int idx = task >> 1, h = task & 1;
        if (idx < Nt) {
          const int i = jn + idx;
          T v[NB], o[NB / 2];
#pragma unroll
          for (int k = 0; k < NB; k += 4) ld4(&S[(size_t)i * LDS + j0 + k], &v[k]);
#pragma unroll
          for (int q = 0; q < NB / 2; ++q) {
            const int c = 2 * q + h;
            T s2 = 0;
#pragma unroll
            for (int k = 0; k < NB; k += 4) {
              if (k <= 2 * q + 1) {   // D is zero beyond the diagonal
                T dv[4];
                ld4(&Dinv[c][k], dv);
                s2 += v[k] * dv[0] + v[k + 1] * dv[1] + v[k + 2] * dv[2] + v[k + 3] * dv[3];
              }
            }
            o[q] = s2;
          }
#pragma unroll
          for (int q = 0; q < NB / 2; ++q) {
            const int c = 2 * q + h;
            PT[c * PTLD + i] = o[q];
            S[(size_t)i * LDS + j0 + c] = o[q];
          }
        } else {
          const int c = idx - Nt;
          if (c < j0) {
            T w[NB], o[NB / 2];
#pragma unroll
            for (int k = 0; k < NB; k += 4) ld4(&S[(size_t)c * LDS + j0 + k], &w[k]);
            if (jb < NB) {
#pragma unroll
              for (int k = 0; k < NB; ++k)
                if (k >= jb) w[k] = (T)0;
            }
#pragma unroll
            for (int q = 0; q < NB / 2; ++q) {
              const int rr = 2 * q + h;
              T s2 = 0;
#pragma unroll
              for (int k = 0; k < NB; k += 4) {
                if (k <= 2 * q + 1) {
                  T dv[4];
                  ld4(&Dinv[rr][k], dv);
                  s2 += dv[0] * w[k] + dv[1] * w[k + 1] + dv[2] * w[k + 2] + dv[3] * w[k + 3];
                }
              }
              o[q] = s2;
            }
#pragma unroll
            for (int q = 0; q < NB / 2; ++q) {
              const int rr = 2 * q + h;
              if (rr < jb) {
                S[(size_t)c * LDS + j0 + rr] = o[q];
                WT[rr * PTLD + c] = o[q];
              }
            }
          } else {
            const int cc = c - j0;
            if (h == 0) wdiag[c] = Dinv[cc][cc];
#pragma unroll
            for (int q = 0; q < NB / 2; ++q) {
              const int rr = 2 * q + h;
              if (rr < jb) {
                const T wv = rr >= cc ? Dinv[rr][cc] : (T)0;
                if (rr > cc) S[(size_t)c * LDS + j0 + rr] = wv;
                WT[rr * PTLD + c] = wv;
              }
            }
          }
        }
      }
      __syncthreads();
      // (3) trailing updates G_II -= L_IJ L_IJ^T (lower part) and X -= L_IJ W_J,:
      // (rows above), each thread taking 4 x 4 blocks: two 128-bit loads of
      // panel values per 16 FMAs, then a vectorised read-modify-write of S.
      if (Nt > 0) {
        const int nbc = (Nt + 3) / 4;              // 4-column blocks over [jn, d)
        const int nbl = nbc * (nbc + 1) / 2;       // lower blocks: block row >= block column
        const int nbw = ((jn + 3) / 4) * nbc;      // W blocks: rows [0, jn) x columns [jn, d)
        for (int b = tid; b < nbl + nbw; b += blockDim.x) {
          int r0, c0, rlim;
          bool lower;
          if (b < nbl) {
            int br = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
            while ((br + 1) * (br + 2) / 2 <= b) ++br;
            while (br * (br + 1) / 2 > b) --br;
            r0 = jn + 4 * br;
            c0 = jn + 4 * (b - br * (br + 1) / 2);
            rlim = d;
            lower = true;
          } else {
            const int w = b - nbl;
            r0 = 4 * (w / nbc);
            c0 = jn + 4 * (w % nbc);
            rlim = jn;
            lower = false;
          }
          const T* Ar = lower ? PT : WT;
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
    float* r = R + (int64_t)i * ldr;
    float* ri = Rinv + (int64_t)i * ldr;
    for (int l = lane; l < d; l += 32) {
      r[l] = l >= i ? (float)S[(size_t)l * LDS + i] : 0.f;
      ri[l] = l > i ? (float)S[(size_t)i * LDS + l] : (l == i ? (float)wdiag[i] : 0.f);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
chol_blocked_kernel(int d, const float* __restrict__ G, int64_t ldg, float* __restrict__ R, float* __restrict__ Rinv,
                    int64_t ldr, int* info, double* shift_count, int* gate_out, const int* gate_in, T* gS) {
  chol_body<T>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in, gS);
}

// One CTA per problem of a batch; every square buffer in shared memory.
template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 3)
chol_batched_kernel(const CholJob* __restrict__ jobs, int count) {
  const int b = blockIdx.x;
  if (b >= count) return;
  const CholJob j = jobs[b];
  chol_body<T>(j.d, j.G, j.ldg, j.R, j.Rinv, j.ldr, j.info, j.shift_count, j.gate_out, j.gate_in, nullptr);
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
size_t static_bytes() { return (2 * kMaxD + NB * NB + NB + 32) * sizeof(T) + 96; }
template <typename T>
bool square_in_smem(int d) {
  return square_bytes<T>(d) + panel_bytes<T>(d) + static_bytes<T>() <= smem_optin_chol();
}

template <typename T>
cudaError_t launch(int d, const float* G, int64_t ldg, float* R, float* Rinv, int64_t ldr, int* info,
                   double* shift_count, int* gate_out, const int* gate_in, void* gstore, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(chol_blocked_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem_optin_chol() - static_bytes<T>()));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const bool in_smem = square_in_smem<T>(d);
  if (!in_smem && gstore == nullptr) return cudaErrorInvalidValue;
  const size_t dyn = panel_bytes<T>(d) + (in_smem ? square_bytes<T>(d) : 0);
  chol_blocked_kernel<T><<<1, kThreads, dyn, st>>>(d, G, ldg, R, Rinv, ldr, info, shift_count, gate_out, gate_in,
                                                    in_smem ? nullptr : reinterpret_cast<T*>(gstore));
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
