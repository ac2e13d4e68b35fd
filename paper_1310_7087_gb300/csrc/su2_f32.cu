// su2_f32.cu -- kernels of the gauge sweep for SU(2) with FP32 4-real links (quaternions).
// The phase update uses the kernels of qcd_su2c.cuh; reunitarization, start,
// measurements and layout conversion use the shared templates.
#include "qcd_su2c.cuh"

namespace qcd {
const PolicyOps kOpsSU2F32 = su2c_ops<float>(1);
}  // namespace qcd
