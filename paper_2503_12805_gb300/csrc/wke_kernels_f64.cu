// Double-precision instantiation of the kernels.  The fused axis-0 + product
// kernel is single precision only; its double launchers return an error.
#include "wke_launch.cuh"

namespace wke {
template WKE_FUSED_AT(double, 16)
template WKE_FUSED_AT(double, 32)
template WKE_FUSED_AT(double, 48)
template WKE_FUSED_AT(double, 64)
WKE_INSTANTIATE(double)
int check_bind_kernels_f64() { return check_bind(); }
}  // namespace wke
