// cm_bwd_k8.cu -- the adjoint kernel's builds for K <= 8 (see cm_bwd.cuh).
#include "cm_bwd.cuh"

namespace cm {

template cudaError_t launch_bwd_t<1, 8>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);
template cudaError_t launch_bwd_t<2, 8>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);

}  // namespace cm
