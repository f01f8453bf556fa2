// FP64 instantiations of the 3D kernels (Cartesian, first order, 0-3 passive scalars).
#include "roeam3_kernels.cuh"

namespace roeam {
template struct Launchers3<double>;
}
