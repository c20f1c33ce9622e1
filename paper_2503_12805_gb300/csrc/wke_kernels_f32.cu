// Single-precision instantiation of the kernels (transforms and products in
// float; forward transform, group sums and tables in double).
#include "wke_launch.cuh"

namespace wke {
WKE_INSTANTIATE(float)
}  // namespace wke
