// Tensor-core passes over A (BF16 split precision). Not yet available: the
// entry points report the option as unsupported.
#include "tc_gemm.cuh"

namespace rqlp {

bool tc_supported(const float*, int64_t, const float*, int64_t) { return false; }

void TcEngine::layout(Arena&, int64_t, int64_t, int) {}

cudaError_t TcEngine::pass(bool, const float*, int64_t, int64_t, int64_t, const float*, int64_t, int, float*,
                           int64_t, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace rqlp
