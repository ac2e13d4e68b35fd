// su2_f32.cu -- kernels of the gauge sweep instantiated for one (group, storage).
#include "qcd_kernels.cuh"

namespace qcd {
const PolicyOps kOpsSU2F32 = make_ops<SU2Policy<float>>(1);
}  // namespace qcd
