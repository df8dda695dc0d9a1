// fx_stream.cuh -- the streaming fast path (device code).  Placeholder until
// the specialised kernel lands: routes every unit to the general tile.
#pragma once
#include "fx_internal.h"
#include "fx_tile.cuh"

namespace fx {

constexpr int kDefaultUnitW = gen::TW;
constexpr int kDefaultUnitH = gen::TH;
constexpr int kNumUnitShapes = 1;
constexpr int kUnitShapes[kNumUnitShapes][2] = {{gen::TW, gen::TH}};
constexpr int kMaxCtasPerSm = 4;

inline bool fast_unit_shape_ok(int w, int h) { return w == gen::TW && h == gen::TH; }

inline size_t fast_smem_bytes(int r_in, int, int) {
  KParams kp{};
  kp.r_m = r_in - 5;
  return gen::general_smem_bytes(kp);
}

template <typename T>
__device__ void fast_unit(const ImageView &v, const KParams &kp, int64_t ux, int64_t uy, int uw, int uh,
                          unsigned char *smem) {
  gen::general_tile<T>(v, kp, ux * gen::TW, uy * gen::TH, smem);
}

}  // namespace fx
