// Bounds checks of the bounds-checked debug build (compiled with -DWKE_CHECK).
//
// In a checked build the hot kernels test the indices they derive from the
// plan's tables (plane and pair ids, field slots, schedule offsets, unit
// numbers) against the extents of the buffers they address.  A failed test
// records a bit naming the check site in a device word and skips the access;
// nothing traps, so the context stays usable, and wke_check_status() reads
// and clears the word (returning WKE_ERR_CUDA when a bit is set).  Each
// translation unit holds its own copy of the word's address in constant
// memory, bound once per device before its first checked launch.  In the
// default build every check compiles to nothing.
#pragma once

#include <cuda_runtime.h>

namespace wke {

// Check sites (bits of the device word).
enum CheckSite : unsigned {
    kChkFusedPlane = 1u << 0,     // fused kernel: staged plane / unit index
    kChkFusedSchedule = 1u << 1,  // fused kernel: product-schedule offset outside the field slots
    kChkSepPair = 1u << 2,        // separable pass: row value, pair or field id
    kChkProductsSlot = 1u << 3,   // product pass: field slot or table id
    kChkAxis0Unit = 1u << 5,      // axis-0 pass: unit or pair id
};

// Address of the current device's check word (allocated on first use;
// nullptr if that fails).  Defined in wke_api.cu.
unsigned *check_word();

// Bind the check word in each kernel translation unit on the current device
// (checked builds; a no-op returning 0 otherwise).  Called at plan creation,
// outside any stream capture: the binding copies to constant memory.
int check_bind_kernels_f32();
int check_bind_kernels_f64();
int check_bind_fused64_f32();
int check_bind_fused_f32();

#ifdef WKE_CHECK
static __constant__ unsigned *c_wke_check = nullptr;

// Bind this translation unit's copy of the word's address on the current
// device (once per device).
static inline int check_bind() {
    static unsigned *bound[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
    if (bound[dev]) return 0;
    unsigned *w = check_word();
    if (!w) return (int)cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemcpyToSymbol(c_wke_check, &w, sizeof(w));
    if (e != cudaSuccess) return (int)e;
    bound[dev] = w;
    return 0;
}

// True when `ok`; otherwise records `site` and returns false.
__device__ __forceinline__ bool wke_guard(bool ok, unsigned site) {
    if (!ok && c_wke_check) atomicOr(c_wke_check, site);
    return ok;
}
#define WKE_GUARD(cond, site) ::wke::wke_guard((cond), (site))
#else
static inline int check_bind() { return 0; }
#define WKE_GUARD(cond, site) true
#endif

}  // namespace wke
