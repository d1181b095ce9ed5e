// cm_bwd.cu -- dispatch of the adjoint kernel builds (instantiated in
// cm_bwd_k8.cu, cm_bwd_k8b.cu, cm_bwd_k16.cu and cm_bwd_k16b.cu, see cm_bwd.cuh).
#include "cm_bwd.cuh"

namespace cm {

extern template cudaError_t launch_bwd_t<1, 8>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);
extern template cudaError_t launch_bwd_t<2, 8>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);
extern template cudaError_t launch_bwd_t<1, 16>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);
extern template cudaError_t launch_bwd_t<2, 16>(const FwdArgs&, const float*, float*, float*, int, int, cudaStream_t);
int bwd_occupancy_1(int block, int smem_bytes);
int bwd_occupancy_2(int block, int smem_bytes);

cudaError_t launch_bwd(const FwdArgs& a, const float* grad_out, float* grad_poses, float* grad_dims, int grid,
                       int block, int per_sm, cudaStream_t s) {
  const bool k8 = a.p.K <= 8;
  if (per_sm == 1 || a.sm.total > kBwdSmem2)
    return k8 ? launch_bwd_t<1, 8>(a, grad_out, grad_poses, grad_dims, grid, block, s)
              : launch_bwd_t<1, 16>(a, grad_out, grad_poses, grad_dims, grid, block, s);
  return k8 ? launch_bwd_t<2, 8>(a, grad_out, grad_poses, grad_dims, grid, block, s)
            : launch_bwd_t<2, 16>(a, grad_out, grad_poses, grad_dims, grid, block, s);
}

int bwd_max_blocks_per_sm(int block, int smem_bytes, int per_sm) {
  return (per_sm == 1 || smem_bytes > kBwdSmem2) ? bwd_occupancy_1(block, smem_bytes)
                                                 : bwd_occupancy_2(block, smem_bytes);
}

}  // namespace cm
