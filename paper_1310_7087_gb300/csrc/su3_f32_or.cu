// su3_f32_or.cu -- the SU(3) FP32 overrelaxation kernels that also
// reunitarize each link they update (the last pass of a sweep), in a
// translation unit of their own so they compile in parallel with su3_f32.cu.
#include "qcd_su3c.cuh"

namespace qcd {
cudaError_t su3c_launch_or_reunit(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  su3c_launch_level<KIND_OR_REUNIT>(a, parity, mu, block, st);
  return cudaGetLastError();
}

int su3c_or_reunit_max_block() {
  return std::min(std::min(su3c_block_limit_mu<0, KIND_OR_REUNIT>(), su3c_block_limit_mu<1, KIND_OR_REUNIT>()),
                  su3c_block_limit_mu<2, KIND_OR_REUNIT>());
}
}  // namespace qcd
