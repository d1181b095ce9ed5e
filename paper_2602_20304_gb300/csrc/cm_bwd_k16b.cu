// cm_bwd_k16b.cu -- the adjoint kernel's two-CTAs-per-SM build for K <= 16 (see
// cm_bwd.cuh) and its occupancy.
#include "cm_bwd.cuh"

namespace cm {

template cudaError_t launch_bwd_t<2, 16>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);

int bwd_occupancy_2(int block, int smem_bytes) {
  int n = 0;
  const void* k = reinterpret_cast<const void*>(cm_bwd_kernel<2, 16>);
  if (ensure_smem_attr(k, kBwdSmem2) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cm_bwd_kernel<2, 16>, block, smem_bytes) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace cm
