// Double-precision instantiation of the kernels.
#include "wke_launch.cuh"

namespace wke {
WKE_INSTANTIATE(double)
}  // namespace wke
