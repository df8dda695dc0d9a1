// fx_tile.cu -- grid launch of the general fused extraction tile (fx_tile.cuh).
#include <atomic>

#include "fx_tile.cuh"

namespace fx {
namespace {

using gen::TW;
using gen::TH;
using gen::NT;

template <typename T>
__global__ void __launch_bounds__(NT) tile_general_kernel(ImageView v, KParams kp, int64_t tiles_x) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  gen::general_tile<T>(v, kp, tx * TW, v.y_begin + ty * TH, smem);
}

// The kernel's dynamic shared-memory limit is a per-device attribute: set it
// once on every device the process launches it on.
constexpr int kMaxDevices = 64;

template <typename T>
cudaError_t launch_t(const ImageView &v, const KParams &kp, cudaStream_t s) {
  size_t smem = gen::general_smem_bytes(kp);
  static std::atomic<bool> attr_set[kMaxDevices];  // per template instance and device (idempotent)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || !attr_set[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(tile_general_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) attr_set[dev].store(true, std::memory_order_release);
  }
  int64_t tiles_x = (v.width + TW - 1) / TW;
  int64_t tiles_y = (v.y_end - v.y_begin + TH - 1) / TH;
  int64_t blocks = tiles_x * tiles_y;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  tile_general_kernel<T><<<static_cast<unsigned>(blocks), NT, smem, s>>>(v, kp, tiles_x);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_general(const ImageView &v, const KParams &kp, cudaStream_t s) {
  return v.elem == 1 ? launch_t<uint8_t>(v, kp, s) : launch_t<uint16_t>(v, kp, s);
}

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_tile)
}  // namespace fx
