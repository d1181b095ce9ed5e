// cm_bwd_k8b.cu -- the adjoint kernel's two-CTAs-per-SM build for K <= 8 (see cm_bwd.cuh).
#include "cm_bwd.cuh"

namespace cm {

template cudaError_t launch_bwd_t<2, 8>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);

}  // namespace cm
