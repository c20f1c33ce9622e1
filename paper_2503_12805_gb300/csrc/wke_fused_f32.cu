// Single-precision fused axis-0 + product launchers for N = 16, 32 and 48.
#include "wke_launch.cuh"

namespace wke {
template WKE_FUSED_AT(float, 16)
template WKE_FUSED_AT(float, 32)
template WKE_FUSED_AT(float, 48)
int check_bind_fused_f32() { return check_bind(); }
}  // namespace wke
