// Adjoint kernels of the decoupled Fourier pose search.
#include "common.cuh"

namespace fmbym {

cudaError_t launch_backward(const DevPlan&, const Ws&, int, const long long*, const float*, const float*,
                            const float*, float*, float*, cudaStream_t) {
    return cudaErrorNotSupported;
}

cudaError_t prepare_backward_kernels() { return cudaSuccess; }

}  // namespace fmbym
