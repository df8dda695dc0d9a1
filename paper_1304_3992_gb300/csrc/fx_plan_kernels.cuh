// fx_plan_kernels.cuh -- the batched path's descriptor table and its
// streaming group kernels for one strip class.  Included by fx_plan.cu
// (narrow strips), fx_plan_compact.cu, fx_plan_wide.cu and fx_plan_xwide.cu,
// so the classes compile in parallel; the kernels have internal linkage and
// each class exports its kernel selectors (plan_fast_kernel_*,
// plan_redo_kernel_*).
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "fx_internal.h"
#include "fx_stream.cuh"

namespace fx {

struct BatchImage {
  const void *img;
  int64_t width, height, pitch;
  uint8_t *out;
  int64_t out_pitch;
  int64_t units_x;     // work units across the image
  int64_t unit_begin;  // first queue index of this image
  int32_t elem;
  int32_t pad;
};

// Streaming path: the queue holds four groups of images, in this order: read
// with one aligned load per lane (uint16, uint8), then pixel by pixel (uint16,
// uint8).  Group g owns the units [group_end[g-1], group_end[g]) (group_end[-1]
// = 0) and runs in a kernel of its own.
constexpr int kGroups = 4;
__host__ __device__ constexpr int group_of(bool pair, int elem) { return (pair ? 0 : 2) + (elem == 1 ? 1 : 0); }

struct BatchHeader {
  int64_t total_units;
  int64_t group_end[kGroups];  // streaming path only
  int32_t n;
  int32_t unit_w, unit_h;  // unit shape in output pixels
  int32_t pad;
};

inline size_t table_bytes(int max_images) { return sizeof(BatchHeader) + sizeof(BatchImage) * max_images; }

// Status bits written by the batch kernel.
constexpr int kStatusBadDescriptor = 1;

// Persistent kernels: CTAs (general tile) or warps (streaming strip) pop work
// units -- one output tile / strip segment of one image -- from a global
// counter until the queue is empty.  Units of different images and dtypes
// interleave freely; the image is found by binary search over unit offsets.
__device__ inline int find_image(const BatchImage *ims, int n, long long u) {
  int lo = 0, hi = n - 1;  // last image whose first unit is <= u
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ims[mid].unit_begin <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ inline ImageView view_of(const BatchImage &b) {
  return ImageView{b.img, b.width, b.height, b.pitch, 0, b.elem, b.out, b.out_pitch, 0, b.height, b.height};
}

#ifndef __CUDACC_RTC__
// The streaming kernels of the batched path for one strip class: group g's
// first pass and the redo pass, for a plan's parameters.
const void *plan_fast_kernel(int rm_class, const KParams &kp, int g);
const void *plan_redo_kernel(int rm_class, const KParams &kp);
// group kernel compiled at run time for kp (fx_specialize), or nullptr (fx_jit.cpp)
const void *specialized_batch_kernel(const KParams &kp, int elem, bool pair, int rm_class);
#endif

// One group of the streaming path (load path kPair, pixel type T): its units
// from counter[g].  Each group is a kernel of its own, so a kernel holds one
// strip loop (the register allocation and instruction working set of the
// single-image kernel).
// Cst: as for fx_extract's first pass (RuntimeConsts, or the constants of a
// kernel compiled at run time for one parameter set).
template <typename T, bool kF32Log, bool kPair, bool kSd2, bool kSrcZ, int kRm, class Cst = RuntimeConsts>
__global__ void __launch_bounds__(32 * kWarpsPerCta, kBatchCtas) batch_kernel_fast(const unsigned char *table,
                                                                      unsigned long long *counter, int *status,
                                                                      const __grid_constant__ KParams kp) {
  __shared__ StripWords words;
  constexpr int g = group_of(kPair, sizeof(T));
  const BatchHeader *hdr = reinterpret_cast<const BatchHeader *>(table);
  const BatchImage *ims = reinterpret_cast<const BatchImage *>(table + sizeof(BatchHeader));
  const long long first = g == 0 ? 0 : hdr->group_end[g - 1];
  const long long end = hdr->group_end[g];
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(counter + g, 1ULL);
    const long long u = first + static_cast<long long>(__shfl_sync(0xffffffffu, got, 0));
    if (u >= end) break;
    const BatchImage &b = ims[find_image(ims, hdr->n, u)];
    if (b.units_x <= 0 || b.elem != static_cast<int32_t>(sizeof(T))) {
      if (lane == 0) atomicOr(status, kStatusBadDescriptor);
      continue;
    }
    const ImageView v = view_of(b);
    const long long local = u - b.unit_begin;
    const int64_t ux = local % b.units_x, uy = local / b.units_x;
    fast_unit<T, kF32Log, kPair, kSd2, kSrcZ, false, kRm, Cst>(v, kp, ux, uy, hdr->unit_w, hdr->unit_h,
                                                              warp_words(words));
  }
}

#ifndef __CUDACC_RTC__
namespace {

// Second pass of the streaming path: every warp walks the units with a static
// stride and recomputes, on the integer (or wide FP32-LoG) path, the strips
// the first pass marked.  2 CTAs per SM (no spill of the 64-bit sums); the
// graph launches exactly the resident CTAs, so no CTA waits for a second wave
// with its share of the stride.
template <bool kF32Log, bool kSrcZ, int kRm>
__global__ void __launch_bounds__(32 * kWarpsPerCta, 2) batch_kernel_redo(const unsigned char *table,
                                                                      unsigned long long *, int *,
                                                                      const __grid_constant__ KParams kp8,
                                                                      const __grid_constant__ KParams kp16) {
  __shared__ StripWords words;
  const BatchHeader *hdr = reinterpret_cast<const BatchHeader *>(table);
  const BatchImage *ims = reinterpret_cast<const BatchImage *>(table + sizeof(BatchHeader));
  const long long total = hdr->total_units;
  const long long warps = static_cast<long long>(gridDim.x) * kWarpsPerCta;
  for (long long u = static_cast<long long>(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5); u < total; u += warps) {
    const BatchImage &b = ims[find_image(ims, hdr->n, u)];
    if (b.units_x <= 0 || (b.elem != 1 && b.elem != 2)) continue;
    const ImageView v = view_of(b);
    const long long local = u - b.unit_begin;
    const int64_t ux = local % b.units_x, uy = local / b.units_x;
    if (b.elem == 1) {
      if (kp8.fbound < 0 || kp8.fbound < 255)
        fast_unit_redo<uint8_t, kF32Log, kSrcZ, kRm>(v, kp8, ux, uy, hdr->unit_w, hdr->unit_h, warp_words(words));
    } else {
      fast_unit_redo<uint16_t, kF32Log, kSrcZ, kRm>(v, kp16, ux, uy, hdr->unit_w, hdr->unit_h, warp_words(words));
    }
  }
}

// The streaming kernel of group g for a plan's parameters (LoG mode,
// standard-deviation source and thresholds).
template <typename T, bool kF32Log, bool kPair, int kRm>
const void *fast_kernel_sd(const KParams &kp) {
  if (kp.source == 1) return reinterpret_cast<const void *>(&batch_kernel_fast<T, kF32Log, kPair, false, true, kRm>);
  return kp.sd_same ? reinterpret_cast<const void *>(&batch_kernel_fast<T, kF32Log, kPair, false, false, kRm>)
                    : reinterpret_cast<const void *>(&batch_kernel_fast<T, kF32Log, kPair, true, false, kRm>);
}
template <bool kF32Log, int kRm>
const void *fast_kernel_mode(const KParams &kp, int g) {
  switch (g) {
    case 0: return fast_kernel_sd<uint16_t, kF32Log, true, kRm>(kp);
    case 1: return fast_kernel_sd<uint8_t, kF32Log, true, kRm>(kp);
    case 2: return fast_kernel_sd<uint16_t, kF32Log, false, kRm>(kp);
    default: return fast_kernel_sd<uint8_t, kF32Log, false, kRm>(kp);
  }
}
template <int kRm>
const void *fast_kernel_of(const KParams &kp, int g) {
  return kp.f32log ? fast_kernel_mode<true, kRm>(kp, g) : fast_kernel_mode<false, kRm>(kp, g);
}
template <bool kF32Log, int kRm>
const void *redo_kernel_src(const KParams &kp) {
  return kp.source == 1 ? reinterpret_cast<const void *>(&batch_kernel_redo<kF32Log, true, kRm>)
                        : reinterpret_cast<const void *>(&batch_kernel_redo<kF32Log, false, kRm>);
}
template <int kRm>
const void *redo_kernel_of(const KParams &kp) {
  return kp.f32log ? redo_kernel_src<true, kRm>(kp) : redo_kernel_src<false, kRm>(kp);
}

}  // namespace
#endif
}  // namespace fx
