// su3_f32.cu -- kernels of the gauge sweep instantiated for one (group, storage).
#include "qcd_kernels.cuh"

namespace qcd {
const PolicyOps kOpsSU3F32 = make_ops<SU3Policy<float>>(1);
}  // namespace qcd
