// FP32 instantiations of the Roe-AM kernels (state and flux arithmetic in float,
// reductions and positivity re-decisions in double).
#include "roeam_kernels.cuh"

namespace roeam {
extern template struct AblationLaunchers<float>;   // in roeam_k32_abl.cu
template struct Launchers<float>;
}
