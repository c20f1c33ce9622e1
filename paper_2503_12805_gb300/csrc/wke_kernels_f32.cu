// Single-precision instantiation of the kernels (transforms and products in
// float; forward transform, group sums and tables in double).  The fused
// axis-0 + product launchers are instantiated in wke_fused64_f32.cu and
// wke_fused_f32.cu.
#include "wke_launch.cuh"

namespace wke {
WKE_EXTERN_FUSED(float)
WKE_INSTANTIATE(float)
int check_bind_kernels_f32() { return check_bind(); }
}  // namespace wke
