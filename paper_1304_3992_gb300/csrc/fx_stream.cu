// fx_stream.cu -- launch of the streaming fast path (placeholder).
#include "fx_stream.cuh"

namespace fx {

bool fast_path_supported(const KParams &) { return false; }

cudaError_t launch_fast(const ImageView &v, const KParams &kp, cudaStream_t s) {
  return launch_tile_general(v, kp, s);
}

}  // namespace fx
