// su3_f32.cu -- kernels of the gauge sweep for SU(3) with FP32 12-real links.
// The phase update uses the two-row kernel of qcd_su3c.cuh; reunitarization,
// start, measurements and layout conversion use the shared templates.
#include "qcd_su3c.cuh"

namespace qcd {
using SU3F = SU3Policy<float>;
const PolicyOps kOpsSU3F32 = PolicyOps{3,
                                       1,
                                       SU3F::COMPS,
                                       &su3c_launch_phase,
                                       &launch_reunit<SU3F>,
                                       &launch_start<SU3F>,
                                       &launch_measure<SU3F>,
                                       &launch_to_canonical<SU3F>,
                                       &launch_from_canonical<SU3F>,
                                       &launch_set_frozen<SU3F>,
                                       &su3c_measure_fused_tail,
                                       &su3c_max_phase_block};
}  // namespace qcd
