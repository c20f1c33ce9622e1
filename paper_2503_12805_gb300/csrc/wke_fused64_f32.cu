// Single-precision fused axis-0 + product launcher for N = 64 (the staged
// kernel k_fused64 and its fallback).
#include "wke_launch.cuh"

namespace wke {
template WKE_FUSED_AT(float, 64)
int check_bind_fused64_f32() { return check_bind(); }
}  // namespace wke
