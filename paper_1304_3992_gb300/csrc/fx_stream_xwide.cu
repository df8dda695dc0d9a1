// fx_stream_xwide.cu -- the extra-wide streaming strips (median lists whose
// radii add up to 8 .. 11), compiled apart from the other classes.
#include "fx_stream_kernels.cuh"

namespace fx {

cudaError_t launch_xwide(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                         int64_t units, int uh) {
  return v.elem == 1 ? launch_t<uint8_t, kXWideRm>(v, kp, s, blocks, units_x, units, uh)
                     : launch_t<uint16_t, kXWideRm>(v, kp, s, blocks, units_x, units, uh);
}

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_stream_xwide)
}  // namespace fx
