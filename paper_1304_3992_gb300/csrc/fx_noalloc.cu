// fx_noalloc.cu -- the batched extraction for callers that cannot allocate.
//
// fx_extract_batch keeps its descriptor table and tile-queue counter in device
// memory that fx_plan_create allocates.  Some callers cannot do that: services
// whose device memory is entirely owned by another allocator (a framework's
// caching pool or a fixed arena), real-time loops that forbid cudaMalloc after
// start-up because it can synchronise the device and fail under
// fragmentation, and plug-ins that are handed buffers but no allocation
// rights.  fx_extract_batch_noalloc serves them: its only scratch is the
// fixed-size array below, which the CUDA module reserves when the library is
// loaded and every GPU that loads it holds until the process exits.  The call
// itself allocates nothing, host or device.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "fx_internal.h"
#include "fx_tile.cuh"

namespace fx {
namespace {

struct NoAllocImage {
  const void *img;
  int64_t width, height, pitch;
  uint8_t *out;
  int64_t out_pitch;
  int64_t units_x;
  int64_t unit_begin;
  int32_t elem;
  int32_t pad;
};

// The descriptor table travels as a kernel parameter: the launch copies it,
// so the call needs no host staging buffer and no copy of its own.
struct NoAllocTable {
  int64_t total_units;
  int32_t n;
  int32_t pad;
  NoAllocImage im[FX_NOALLOC_MAX_IMAGES];
};

// The kernel's parameters: the table and one KParams per pixel type (CUDA
// allows 32764 bytes of kernel parameters).
static_assert(sizeof(NoAllocTable) + 2 * sizeof(KParams) + 64 <= 32764, "kernel parameters too large");

// The scratch of every fx_extract_batch_noalloc call on a device: the
// tile-queue counter, reset to zero by each call before its kernel runs.
// Host code must not pass this name to a kernel or a copy: on the host it is
// only a stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress.
constexpr size_t kScratchBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];
bool g_attr_set[kMaxDevices];

// Per-device set-up, once per device with that device current: the scratch
// array's device address and the kernel's dynamic shared-memory limit.
fx_status setup_device(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FX_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FX_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FX_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FX_OK;
}

// The persistent tile-queue loop of the batched path: the table from the
// kernel parameter, the queue counter from the scratch array.
__global__ void __launch_bounds__(gen::NT) noalloc_batch_kernel(unsigned long long *counter,
                                                                 const __grid_constant__ NoAllocTable tab,
                                                                 const __grid_constant__ KParams kp8,
                                                                 const __grid_constant__ KParams kp16) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_unit;
  for (;;) {
    if (threadIdx.x == 0) s_unit = static_cast<long long>(atomicAdd(counter, 1ULL));
    __syncthreads();
    const long long u = s_unit;
    __syncthreads();
    if (u >= tab.total_units) break;
    int lo = 0, hi = tab.n - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (tab.im[mid].unit_begin <= u) lo = mid;
      else hi = mid - 1;
    }
    const NoAllocImage &b = tab.im[lo];
    const long long local = u - b.unit_begin;
    ImageView v{b.img, b.width, b.height, b.pitch, 0, b.elem, b.out, b.out_pitch, 0, b.height, b.height};
    const int64_t ux = local % b.units_x, uy = local / b.units_x;
    if (b.elem == 1) gen::general_tile<uint8_t>(v, kp8, ux * gen::TW, uy * gen::TH, smem);
    else gen::general_tile<uint16_t>(v, kp16, ux * gen::TW, uy * gen::TH, smem);
    __syncthreads();
  }
}

bool overlaps(uintptr_t a0, uintptr_t a1, uintptr_t b0, uintptr_t b1) { return a0 < b1 && b0 < a1; }

}  // namespace
}  // namespace fx

using namespace fx;

extern "C" fx_status fx_extract_batch_noalloc(const fx_params *params, const fx_image_desc *descs,
                                              int32_t n, void *stream) {
  NvtxRange range("fx_extract_batch_noalloc");
  if (!descs || n < 1) return FX_ERR_INVALID_ARG;
  if (n > FX_NOALLOC_MAX_IMAGES) return FX_ERR_BUDGET;
  fx_params def;
  if (!params) {
    fx_params_default(&def, FX_U16, 0);
    params = &def;
  }
  if (params->struct_size != sizeof(fx_params)) return FX_ERR_INVALID_ARG;
  KParams kp8, kp16;
  fx_status st = make_kparams(params, 255, &kp8);
  if (st != FX_OK) return st;
  const fx_status st16 = make_kparams(params, 65535, &kp16);
  if (st16 != FX_OK) kp16 = kp8;

  // The table is filled on the host stack and handed to the launch by value.
  static_assert(sizeof(NoAllocTable) <= 16384, "table on the stack");
  NoAllocTable tab;
  std::memset(&tab, 0, sizeof(tab));
  int64_t total = 0;
  for (int32_t i = 0; i < n; ++i) {
    const fx_image_desc &d = descs[i];
    const int64_t op = d.out_pitch ? d.out_pitch : d.width;
    st = check_image(d.img, d.width, d.height, d.pitch_bytes, d.dtype, d.out_mask, op);
    if (st != FX_OK) return st;
    if (d.dtype == FX_U16 && st16 != FX_OK) return st16;
    NoAllocImage &b = tab.im[i];
    b.img = d.img;
    b.width = d.width;
    b.height = d.height;
    b.pitch = d.pitch_bytes;
    b.out = d.out_mask;
    b.out_pitch = op;
    b.elem = d.dtype == FX_U8 ? 1 : 2;
    b.units_x = (d.width + gen::TW - 1) / gen::TW;
    b.unit_begin = total;
    total += b.units_x * ((d.height + gen::TH - 1) / gen::TH);
  }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) {
      if (i == j) continue;
      const uintptr_t o0 = reinterpret_cast<uintptr_t>(tab.im[i].out);
      const uintptr_t o1 = o0 + (tab.im[i].height - 1) * tab.im[i].out_pitch + tab.im[i].width;
      const uintptr_t p0 = reinterpret_cast<uintptr_t>(tab.im[j].out);
      const uintptr_t p1 = p0 + (tab.im[j].height - 1) * tab.im[j].out_pitch + tab.im[j].width;
      const uintptr_t q0 = reinterpret_cast<uintptr_t>(tab.im[j].img);
      const uintptr_t q1 = q0 + (tab.im[j].height - 1) * tab.im[j].pitch + tab.im[j].width * tab.im[j].elem;
      if ((j > i && overlaps(o0, o1, p0, p1)) || overlaps(o0, o1, q0, q1)) return FX_ERR_INVALID_ARG;
    }
  tab.total_units = total;
  tab.n = n;

  void *scratch = nullptr;
  if ((st = setup_device(&scratch)) != FX_OK) return st;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FX_ERR_CUDA;
  const size_t smem = gen::general_smem_bytes(kp8) > gen::general_smem_bytes(kp16)
                          ? gen::general_smem_bytes(kp8)
                          : gen::general_smem_bytes(kp16);
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_attr_set[dev]) {  // the largest dynamic shared memory any parameter set needs
      if (cudaFuncSetAttribute(noalloc_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
          cudaSuccess)
        return FX_ERR_CUDA;
      g_attr_set[dev] = true;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long *counter = static_cast<unsigned long long *>(scratch);
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s) != cudaSuccess) return FX_ERR_CUDA;
  noalloc_batch_kernel<<<static_cast<unsigned>(sms * 2), gen::NT, smem, s>>>(counter, tab, kp8, kp16);
  return cudaGetLastError() == cudaSuccess ? FX_OK : FX_ERR_CUDA;
}

namespace fx {
FX_CHECK_COUNTER(checked_count_noalloc)
}  // namespace fx
