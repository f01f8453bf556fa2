// FP64 instantiations of the ablation-variant stage kernels (classical Roe with the
// entropy fix of Eqs. 114-115, and Roe-AM without Eq. 92, with xi = |U| or with delta U_p
// = 0 / the Roe form), kept apart so that they compile in parallel with the main kernels.
#include "roeam_kernels.cuh"

namespace roeam {
template struct AblationLaunchers<double>;
}
