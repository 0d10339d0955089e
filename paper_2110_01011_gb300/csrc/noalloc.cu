// rqlp_factor_noalloc: the factorisation for callers that cannot allocate
// device memory.
//
// rqlp_factor needs a caller-provided workspace. Some callers cannot obtain
// one: code that runs inside a framework or host application that owns every
// byte of device memory through its own pool, code with a fixed device-memory
// budget set at start-up, and code on paths where cudaMalloc's implicit device
// synchronisation is not acceptable. For them this entry point takes its
// scratch from one fixed array in device memory that belongs to the library
// (g_noalloc_scratch below, RQLP_NOALLOC_SCRATCH_BYTES bytes). Every GPU that
// loads the library holds that array until the process exits.
//
// Properties:
//  - It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
//    routine. The caller still passes A, Omega and the output buffers.
//  - Problems whose workspace (rqlp_workspace_bytes) exceeds the array are
//    rejected with RQLP_ERR_WORKSPACE before anything is enqueued.
//  - All calls on a device share the one array, which keeps the contents the
//    last call left. Everything the factorisation needs at zero (status
//    words, gate flags, accumulated sums) is cleared by the first kernel of
//    each call; the rest of the scratch is written before it is read.
//  - Calls whose GPU work overlaps (for example on two streams without an
//    ordering between them) race on the array and corrupt each other's
//    results: order them on one stream or with events.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current, so make the first
//    call on each device before starting any stream capture.
#include <mutex>

#include "common.cuh"

namespace rqlp {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RQLP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device). In host code the symbol is only a host-side stand-in, never a
// usable device address, so it is never passed to a kernel directly.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (p == nullptr) return cudaErrorInvalidSymbol;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rqlp

extern "C" rqlp_status rqlp_factor_noalloc(const float* A, int64_t m, int64_t n, int64_t lda, int k, int p,
                                           int q, const float* Omega, int64_t ldo, float* Q, int64_t ldq,
                                           float* L, int64_t ldl, float* P, int64_t ldp, int* d_info,
                                           double* d_diag, const rqlp_opts* opts, void* stream) {
  const size_t need = rqlp_workspace_bytes(m, n, k, p, q, opts);
  if (need == 0) return RQLP_ERR_ARG;
  if (need > (size_t)RQLP_NOALLOC_SCRATCH_BYTES) return RQLP_ERR_WORKSPACE;
  void* scratch = nullptr;
  if (rqlp::scratch_address(&scratch) != cudaSuccess) return RQLP_ERR_CUDA;
  return rqlp_factor(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp, scratch,
                     (size_t)RQLP_NOALLOC_SCRATCH_BYTES, d_info, d_diag, opts, stream);
}
