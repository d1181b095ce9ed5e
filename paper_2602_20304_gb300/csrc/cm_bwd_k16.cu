// cm_bwd_k16.cu -- the adjoint kernel's builds for K <= 16 (see cm_bwd.cuh), and
// the occupancy of a build (the K <= 16 builds bound the K <= 8 ones).
#include "cm_bwd.cuh"

namespace cm {

template cudaError_t launch_bwd_t<1, 16>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);
template cudaError_t launch_bwd_t<2, 16>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);

// CTAs per SM of the one-CTA (mb = 1) or two-CTA (mb = 2) build at this shape.
int bwd_occupancy(int mb, int block, int smem_bytes) {
  int n = 0;
  const void* k = mb == 1 ? reinterpret_cast<const void*>(cm_bwd_kernel<1, 16>)
                          : reinterpret_cast<const void*>(cm_bwd_kernel<2, 16>);
  if (ensure_smem_attr(k, mb == 1 ? kBwdSmem1 : kBwdSmem2) != cudaSuccess) return 1;
  const cudaError_t e =
      mb == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cm_bwd_kernel<1, 16>, block, smem_bytes)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cm_bwd_kernel<2, 16>, block, smem_bytes);
  if (e != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace cm
