// fx_stream.cu -- grid launch of the streaming fast path (fx_stream.cuh).
#include <cstdint>

#include "fx_stream.cuh"

namespace fx {
namespace {

// The first pass runs 3 CTAs (12 warps) per SM in 168 registers; the redo
// pass (64-bit sums) runs 2 per SM, where it needs no spill.
template <typename T, bool kRedoPass, bool kF32Log, bool kPair, bool kSd2, bool kSrcZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, kRedoPass ? 2 : kFirstPassCtas) stream_kernel(const __grid_constant__ ImageView v,
                                                                  const __grid_constant__ KParams kp,
                                                                  int64_t units_x, int64_t units, int uh) {
  __shared__ StripWords words;
  const int64_t unit = static_cast<int64_t>(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
  if (unit >= units) return;  // whole warps only
  if constexpr (kRedoPass)
    fast_unit_redo<T, kF32Log, kSrcZ>(v, kp, unit % units_x, unit / units_x, 0, uh, warp_words(words));
  else
    fast_unit<T, kF32Log, kPair, kSd2, kSrcZ>(v, kp, unit % units_x, unit / units_x, 0, uh, warp_words(words));
}

template <typename T, bool kF32Log, bool kPair>
void launch_first(const ImageView &v, const KParams &kp, cudaStream_t s, unsigned g, int64_t units_x,
                  int64_t units, int uh) {
  constexpr int nt = 32 * kWarpsPerCta;
  if (kp.source == 1) stream_kernel<T, false, kF32Log, kPair, false, true><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
  else if (kp.sd_same) stream_kernel<T, false, kF32Log, kPair, false, false><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
  else stream_kernel<T, false, kF32Log, kPair, true, false><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
}

template <typename T, bool kF32Log>
void launch_mode(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                 int64_t units, int uh) {
  const unsigned g = static_cast<unsigned>(blocks);
  constexpr int nt = 32 * kWarpsPerCta;
  if (kp.fbound >= 0) {
    if (pair_loads_ok(v)) launch_first<T, kF32Log, true>(v, kp, s, g, units_x, units, uh);
    else launch_first<T, kF32Log, false>(v, kp, s, g, units_x, units, uh);
  }
  // the second pass recomputes the strips the first one marked (all when fbound < 0)
  if (kp.fbound < 0 || kp.fbound < (sizeof(T) == 1 ? 255 : 65535)) {
    if (kp.source == 1) stream_kernel<T, true, kF32Log, false, true, true><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
    else stream_kernel<T, true, kF32Log, false, true, false><<<g, nt, 0, s>>>(v, kp, units_x, units, uh);
  }
}

template <typename T>
cudaError_t launch_t(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                     int64_t units, int uh) {
  if (kp.f32log) launch_mode<T, true>(v, kp, s, blocks, units_x, units, uh);
  else launch_mode<T, false>(v, kp, s, blocks, units_x, units, uh);
  return cudaGetLastError();
}

}  // namespace

// The streaming kernel covers both standard-deviation sources and up to two
// median passes whose radii add up to at most 3 (its halo: 2 LoG + 1 crossing
// (+ 2 crossing-map deviation) + 3 median columns).
bool fast_path_supported(const KParams &kp) { return kp.nhmf <= 1 || (kp.nhmf == 2 && kp.r_m <= 3); }

// One aligned load per lane and row: base and pitch multiples of two pixels,
// and an even width or a row pitch with room for one more pixel, so that
// every lane's clamped columns lie in one aligned pair (for an odd width the
// last column's pair also holds the first padding element, which is never
// used; the pair is one aligned load that contains an image element, so it
// stays within the page of that element).
bool pair_loads_ok(const ImageView &v) {
  const int64_t two = 2 * static_cast<int64_t>(v.elem);
  return reinterpret_cast<uintptr_t>(v.img) % two == 0 && v.pitch % two == 0 &&
         (v.width % 2 == 0 || v.pitch >= (v.width + 1) * v.elem);
}

// Resident warps of the streaming kernel on the current device (3 CTAs of 4
// warps per SM), cached per device.
int64_t warp_slots() {
  static int64_t slots[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152 * 12;
  if (!slots[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    slots[dev] = static_cast<int64_t>(sms) * kFirstPassCtas * kWarpsPerCta;
  }
  return slots[dev];
}

// Unit height (rows per warp) for an image of `rows` output rows and `units_x`
// strips: a unit computes about uh + overhead rows (ring prefill, the rows
// above its first output and the rows below its last one that outputs need),
// and the launch takes about ceil(units / resident warps) unit times, so small
// images get short units (parallelism) and large ones long units.  Heights are
// multiples of 16 up to 768.
int unit_height(int64_t rows, int64_t units_x, const KParams &kp) {
  const int64_t slots = warp_slots();
  const int64_t overhead = 20 + kp.r_m + (kp.source == 1 ? 2 : 0);
  int best = 768;
  int64_t best_cost = INT64_MAX;
  for (int uh = 768; uh >= 16; uh -= 16) {
    const int64_t units = units_x * ((rows + uh - 1) / uh);
    const int64_t cost = (units + slots - 1) / slots * (uh + overhead);
    if (cost < best_cost) {
      best_cost = cost;
      best = uh;
    }
  }
  return best;
}

cudaError_t launch_fast(const ImageView &v, const KParams &kp, cudaStream_t s) {
  const int uw = strip_width(kp.source == 1);
  const int64_t units_x = (v.width + uw - 1) / uw;
  const int uh = unit_height(v.y_end - v.y_begin, units_x, kp);
  const int64_t units_y = (v.y_end - v.y_begin + uh - 1) / uh;
  const int64_t units = units_x * units_y;
  if (units <= 0) return cudaSuccess;
  const int64_t blocks = (units + kWarpsPerCta - 1) / kWarpsPerCta;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  return v.elem == 1 ? launch_t<uint8_t>(v, kp, s, blocks, units_x, units, uh)
                     : launch_t<uint16_t>(v, kp, s, blocks, units_x, units, uh);
}

}  // namespace fx
