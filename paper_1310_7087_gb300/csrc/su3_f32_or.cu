// su3_f32_or.cu -- the SU(3) FP32 overrelaxation kernels that also
// reunitarize each link they update (the last pass of a sweep), in a
// translation unit of their own so they compile in parallel with su3_f32.cu.
#include "qcd_su3c.cuh"

namespace qcd {
cudaError_t su3c_launch_or_reunit(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  su3c_launch_level<KIND_OR_REUNIT>(a, parity, mu, block, st);
  return cudaGetLastError();
}

template <int FIELD, int MU>
inline void launch_or_meas_one(const Ctx& a, int parity, int block, cudaStream_t st) {
  launch_programmatic(su3c_or_meas_kernel<FIELD, MU>, grid_for(a.g.Vh, block), block, st, a, parity);
}

template <int FIELD>
inline void launch_or_meas_mu(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  switch (mu) {
    case 1: launch_or_meas_one<FIELD, 1>(a, parity, block, st); break;
    case 2: launch_or_meas_one<FIELD, 2>(a, parity, block, st); break;
    default: launch_or_meas_one<FIELD, 3>(a, parity, block, st); break;
  }
}

cudaError_t su3c_launch_or_meas(const Ctx& a, int parity, int mu, int block, cudaStream_t st) {
  switch (su3_field_level(a)) {
    case 0: launch_or_meas_mu<0>(a, parity, mu, block, st); break;
    case 1: launch_or_meas_mu<1>(a, parity, mu, block, st); break;
    default: launch_or_meas_mu<2>(a, parity, mu, block, st); break;
  }
  return cudaGetLastError();
}

template <int FIELD, int MU>
int or_meas_limit() {
  cudaFuncAttributes attr{};
  return cudaFuncGetAttributes(&attr, su3c_or_meas_kernel<FIELD, MU>) == cudaSuccess ? attr.maxThreadsPerBlock : 0;
}

template <int FIELD>
int or_meas_limit_mu() {
  return std::min(std::min(or_meas_limit<FIELD, 1>(), or_meas_limit<FIELD, 2>()), or_meas_limit<FIELD, 3>());
}

int su3c_or_reunit_max_block() {
  int m = std::min(std::min(su3c_block_limit_mu<0, KIND_OR_REUNIT>(), su3c_block_limit_mu<1, KIND_OR_REUNIT>()),
                   su3c_block_limit_mu<2, KIND_OR_REUNIT>());
  return std::min(m, std::min(std::min(or_meas_limit_mu<0>(), or_meas_limit_mu<1>()), or_meas_limit_mu<2>()));
}
}  // namespace qcd
