// su3_f64.cu -- kernels of the gauge sweep instantiated for one (group, storage).
#include "qcd_kernels.cuh"

namespace qcd {
const PolicyOps kOpsSU3F64 = make_ops<SU3Policy<double>>(0);
}  // namespace qcd
