// fx_checked.cuh -- range checks of the kernels' memory accesses (the
// FX_CHECKED build).
//
// Compiled with -DFX_CHECKED, every global and shared-memory index of the
// streaming, general tile and grayscale median kernels passes FX_GUARD(ok)
// first: a failed check adds one to a device counter and the access is
// skipped (a load keeps its previous value); nothing traps.  The library is
// built without device-side linking, so each translation unit holds its own
// counter and reads it back through the host function that
// FX_CHECK_COUNTER(name) defines there; fx_checked_violations() sums them.
// In the normal build FX_GUARD(ok) is the constant true and ok is not
// evaluated.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

namespace fx {

#ifdef FX_CHECKED
static __device__ unsigned long long g_fx_check_failures;
__device__ __forceinline__ bool fx_guard(bool ok) {
  if (!ok) atomicAdd(&g_fx_check_failures, 1ULL);
  return ok;
}
#define FX_GUARD(ok) ::fx::fx_guard(ok)
#define FX_CHECK_COUNTER(name)                                                                 \
  unsigned long long name(bool reset) {                                                        \
    unsigned long long h = 0;                                                                  \
    if (cudaMemcpyFromSymbol(&h, g_fx_check_failures, sizeof h) != cudaSuccess) return ~0ULL; \
    if (reset) {                                                                               \
      const unsigned long long z = 0;                                                          \
      if (cudaMemcpyToSymbol(g_fx_check_failures, &z, sizeof z) != cudaSuccess) return ~0ULL;  \
    }                                                                                          \
    return h;                                                                                  \
  }
#else
#define FX_GUARD(ok) true
#define FX_CHECK_COUNTER(name) \
  unsigned long long name(bool) { return 0; }
#endif

}  // namespace fx
