// fx_stream_kernels.cuh -- the streaming kernels and their launch for one
// strip class (compact: median radii up to 1; narrow: up to 3; wide: 4 .. 7;
// extra wide: 8 .. 11).  Included by fx_stream_compact.cu, fx_stream.cu,
// fx_stream_wide.cu and fx_stream_xwide.cu, so the classes compile in
// parallel; every definition has internal linkage.
#pragma once
#include <cstdint>

#include "fx_stream.cuh"

namespace fx {
namespace {

// The redo pass (64-bit sums) runs 2 CTAs per SM, where it needs no spill.
template <typename T, bool kF32Log, bool kSrcZ, int kRm>
__global__ void __launch_bounds__(32 * kWarpsPerCta, 2) stream_redo_kernel(const __grid_constant__ ImageView v,
                                                                            const __grid_constant__ KParams kp,
                                                                            int64_t units_x, int64_t units, int uh) {
  __shared__ StripWords words;
  const int64_t unit = static_cast<int64_t>(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
  if (unit >= units) return;  // whole warps only
  fast_unit_redo<T, kF32Log, kSrcZ, kRm>(v, kp, unit % units_x, unit / units_x, 0, uh, warp_words(words));
}

template <typename T, bool kF32Log, bool kPair, int kRm>
void launch_first(const ImageView &v, const KParams &kp, cudaStream_t s, unsigned g, int64_t units_x,
                  int64_t units, int uh) {
  constexpr int nt = 32 * kWarpsPerCta;
  // a kernel compiled for this parameter set (fx_specialize), if there is one
  if (const void *jk = specialized_kernel(kp, sizeof(T), kPair, kRm)) {
    void *args[] = {const_cast<ImageView *>(&v), const_cast<KParams *>(&kp), &units_x, &units, &uh};
    if (cudaLaunchKernel(jk, dim3(g), dim3(nt), args, 0, s) == cudaSuccess) return;
  }
  using C = RuntimeConsts;
  if (kp.source == 1) stream_kernel<T, kF32Log, kPair, false, true, kRm, C><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
  else if (kp.sd_same) stream_kernel<T, kF32Log, kPair, false, false, kRm, C><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
  else stream_kernel<T, kF32Log, kPair, true, false, kRm, C><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
}

template <typename T, bool kF32Log, int kRm>
void launch_mode(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                 int64_t units, int uh) {
  const unsigned g = static_cast<unsigned>(blocks);
  constexpr int nt = 32 * kWarpsPerCta;
  if (kp.fbound >= 0) {
    if (pair_loads_ok(v)) launch_first<T, kF32Log, true, kRm>(v, kp, s, g, units_x, units, uh);
    else launch_first<T, kF32Log, false, kRm>(v, kp, s, g, units_x, units, uh);
  }
  // the second pass recomputes the strips the first one marked (all when fbound < 0)
  if (kp.fbound < 0 || kp.fbound < (sizeof(T) == 1 ? 255 : 65535)) {
    if (kp.source == 1) stream_redo_kernel<T, kF32Log, true, kRm><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
    else stream_redo_kernel<T, kF32Log, false, kRm><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
  }
}

template <typename T, int kRm>
cudaError_t launch_t(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                     int64_t units, int uh) {
  if (kp.f32log) launch_mode<T, true, kRm>(v, kp, s, blocks, units_x, units, uh);
  else launch_mode<T, false, kRm>(v, kp, s, blocks, units_x, units, uh);
  return cudaGetLastError();
}


}  // namespace
}  // namespace fx
