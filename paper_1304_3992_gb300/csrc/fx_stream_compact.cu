// fx_stream_compact.cu -- the compact streaming strips (no median, or one
// window-3 median: 56 output columns per 64-column window), compiled apart
// from the other classes.
#include "fx_stream_kernels.cuh"

namespace fx {

cudaError_t launch_compact(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                           int64_t units, int uh) {
  return v.elem == 1 ? launch_t<uint8_t, kCompactRm>(v, kp, s, blocks, units_x, units, uh)
                     : launch_t<uint16_t, kCompactRm>(v, kp, s, blocks, units_x, units, uh);
}

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_stream_compact)
}  // namespace fx
