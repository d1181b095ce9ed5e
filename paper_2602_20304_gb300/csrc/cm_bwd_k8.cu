// cm_bwd_k8.cu -- the adjoint kernel's one-CTA-per-SM build for K <= 8 (see
// cm_bwd.cuh); each build is its own translation unit so that they compile in parallel.
#include "cm_bwd.cuh"

namespace cm {

template cudaError_t launch_bwd_t<1, 8>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);

}  // namespace cm
