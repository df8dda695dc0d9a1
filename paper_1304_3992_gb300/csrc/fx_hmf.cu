// fx_hmf.cu -- the hybrid median filter (Sec. 3.4) on uint8 / uint16 images.
//
// Output = median(median of the '+' subgroup, median of the 'x' subgroup,
// centre), the subgroups being the centre row/column segment and the two
// diagonals of the k x k window (2k - 1 values each, k = 3 or 5); pixels
// outside the image take the value of the nearest image pixel (replicated
// borders).  Medians come from exact min/max identities:
//   med3(a, b, c)  = max(min(a, b), min(max(a, b), c))
//   med5           = med3(c, max(min(a, b), min(d, e)), min(max(a, b), max(d, e)))
//   med9 of three triples = med3(max of the triples' minima,
//                                med3 of their medians, min of their maxima)
// One CTA stages its tile plus a 2-pixel halo in shared memory once.
#include <cstdint>

#include "fx_internal.h"

namespace fx {
namespace {

constexpr int HW = 64, HH = 16, HR = 2, HNT = 256;
constexpr int SW = HW + 2 * HR, SH = HH + 2 * HR;

__device__ __forceinline__ int mn(int a, int b) { return a < b ? a : b; }
__device__ __forceinline__ int mx(int a, int b) { return a > b ? a : b; }
__device__ __forceinline__ int med3(int a, int b, int c) { return mx(mn(a, b), mn(mx(a, b), c)); }
__device__ __forceinline__ int med5(int a, int b, int c, int d, int e) {
  return med3(c, mx(mn(a, b), mn(d, e)), mn(mx(a, b), mx(d, e)));
}
// median of {a0..a2} U {b0..b2} U {c0..c2}
__device__ __forceinline__ int med9(int a0, int a1, int a2, int b0, int b1, int b2, int c0, int c1, int c2) {
  const int alo = mn(mn(a0, a1), a2), ahi = mx(mx(a0, a1), a2), amd = a0 + a1 + a2 - alo - ahi;
  const int blo = mn(mn(b0, b1), b2), bhi = mx(mx(b0, b1), b2), bmd = b0 + b1 + b2 - blo - bhi;
  const int clo = mn(mn(c0, c1), c2), chi = mx(mx(c0, c1), c2), cmd = c0 + c1 + c2 - clo - chi;
  return med3(mx(mx(alo, blo), clo), med3(amd, bmd, cmd), mn(mn(ahi, bhi), chi));
}

template <typename T>
__global__ void __launch_bounds__(HNT) hmf_kernel(const T *img, int64_t W, int64_t H, int64_t pitch, T *out,
                                                  int64_t out_pitch, int k, int64_t tiles_x) {
  __shared__ int t[SH][SW + 1];
  const int64_t tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int64_t x0 = tx * HW, y0 = ty * HH;
  for (int i = threadIdx.x; i < SH * SW; i += HNT) {
    const int ly = i / SW, lx = i % SW;
    int64_t x = x0 - HR + lx, y = y0 - HR + ly;
    x = x < 0 ? 0 : (x >= W ? W - 1 : x);
    y = y < 0 ? 0 : (y >= H ? H - 1 : y);
    t[ly][lx] = static_cast<int>(*reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(img) +
                                                              y * pitch + x * sizeof(T)));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < HW * HH; i += HNT) {
    const int ly = i / HW, lx = i % HW;
    const int64_t x = x0 + lx, y = y0 + ly;
    if (x >= W || y >= H) continue;
    const int cy = ly + HR, cx = lx + HR, c = t[cy][cx];
    int plus, cross;
    if (k == 5) {
      plus = med9(t[cy][cx - 2], t[cy][cx - 1], c, t[cy][cx + 1], t[cy][cx + 2], t[cy - 2][cx],
                  t[cy - 1][cx], t[cy + 1][cx], t[cy + 2][cx]);
      cross = med9(t[cy - 2][cx - 2], t[cy - 1][cx - 1], c, t[cy + 1][cx + 1], t[cy + 2][cx + 2],
                   t[cy - 2][cx + 2], t[cy - 1][cx + 1], t[cy + 1][cx - 1], t[cy + 2][cx - 2]);
    } else {
      plus = med5(t[cy][cx - 1], t[cy - 1][cx], c, t[cy + 1][cx], t[cy][cx + 1]);
      cross = med5(t[cy - 1][cx - 1], t[cy - 1][cx + 1], c, t[cy + 1][cx - 1], t[cy + 1][cx + 1]);
    }
    *reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(out) + y * out_pitch + x * sizeof(T)) =
        static_cast<T>(med3(plus, cross, c));
  }
}

}  // namespace
}  // namespace fx

using namespace fx;

extern "C" fx_status fx_hybrid_median(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                                      fx_dtype dtype, int32_t window, void *out, int64_t out_pitch_bytes,
                                      void *stream) {
  if (window != 3 && window != 5) return FX_ERR_INVALID_ARG;
  if (!img || !out || (dtype != FX_U8 && dtype != FX_U16)) return FX_ERR_INVALID_ARG;
  const int64_t elem = dtype == FX_U8 ? 1 : 2;
  if (out_pitch_bytes == 0) out_pitch_bytes = width * elem;
  if (width < 1 || height < 1 || width > (1LL << 30) || height > (1LL << 30)) return FX_ERR_INVALID_ARG;
  if (out_pitch_bytes < width * elem || out_pitch_bytes % elem || reinterpret_cast<uintptr_t>(out) % elem)
    return FX_ERR_INVALID_ARG;
  // the same validation as the extraction, with a mask-sized stand-in for the output check
  fx_status st = check_image(img, width, height, pitch_bytes, dtype, static_cast<const uint8_t *>(out),
                             out_pitch_bytes);
  if (st != FX_OK) return st;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(img), a1 = a0 + (height - 1) * pitch_bytes + width * elem;
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(out), b1 = b0 + (height - 1) * out_pitch_bytes + width * elem;
  if (a0 < b1 && b0 < a1) return FX_ERR_INVALID_ARG;
  const int64_t tiles_x = (width + HW - 1) / HW, tiles = tiles_x * ((height + HH - 1) / HH);
  if (tiles > 0x7fffffffLL) return FX_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == FX_U8)
    hmf_kernel<uint8_t><<<static_cast<unsigned>(tiles), HNT, 0, s>>>(
        static_cast<const uint8_t *>(img), width, height, pitch_bytes, static_cast<uint8_t *>(out), out_pitch_bytes,
        window, tiles_x);
  else
    hmf_kernel<uint16_t><<<static_cast<unsigned>(tiles), HNT, 0, s>>>(
        static_cast<const uint16_t *>(img), width, height, pitch_bytes, static_cast<uint16_t *>(out),
        out_pitch_bytes, window, tiles_x);
  return cudaGetLastError() == cudaSuccess ? FX_OK : FX_ERR_CUDA;
}
