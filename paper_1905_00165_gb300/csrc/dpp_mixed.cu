// Mixed-precision (3xTF32) Hermitian sampler.
#include "dpp_device.cuh"
#include "dpp_internal.h"

namespace dpp {

size_t ws_mixed(int64_t) { return 0; }

cudaError_t sample_mixed(const DrawArgs&, Workspace) { return cudaErrorNotSupported; }

}  // namespace dpp
