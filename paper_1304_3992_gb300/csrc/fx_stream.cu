// fx_stream.cu -- grid launch of the streaming fast path (fx_stream.cuh): the
// narrow strips, the unit height and the load-path choice.
#include <cstdint>

#include "fx_stream_kernels.cuh"

namespace fx {

// The streaming kernels cover both standard-deviation sources and up to four
// median passes: compact strips while the median radii add up to at most 1
// (halo: 2 LoG + 1 crossing (+ 2 crossing-map deviation) + 1 median column),
// narrow strips up to 3, wide strips up to 7, extra-wide strips up to 11.
// The batched plans use the same classes (fx_plan.cu).
bool fast_path_supported(const KParams &kp) { return kp.nhmf <= FX_MAX_HMF_LEVELS && kp.r_m <= kXWideRm; }
int strip_class(const KParams &kp) {
  return kp.r_m <= kCompactRm ? kCompactRm : kp.r_m <= kNarrowRm ? kNarrowRm : kp.r_m <= kWideRm ? kWideRm : kXWideRm;
}

// One aligned load per lane and row: base and pitch multiples of 4 bytes.
// uint16: an even width or a row pitch with room for one more pixel, so that
// every lane's clamped columns lie in one aligned pair (for an odd width the
// last column's pair also holds the first padding element, which is never
// used).  uint8: each lane loads the aligned 4-byte word holding its pair, so
// the row pitch reaches the end of the word that holds the last pair.  Every
// such load starts inside the row, so it stays within the page of an image
// element.
bool pair_loads_ok(const void *img, int64_t width, int64_t pitch, int64_t elem) {
  if (reinterpret_cast<uintptr_t>(img) % 4 != 0 || pitch % 4 != 0) return false;
  if (elem == 2) return width % 2 == 0 || pitch >= (width + 1) * elem;
  const int64_t pair_end = width + (width & 1);  // one past the last pair
  return pitch >= (pair_end + 3) / 4 * 4;
}
bool pair_loads_ok(const ImageView &v) { return pair_loads_ok(v.img, v.width, v.pitch, v.elem); }

// Resident warps of the streaming kernel on the current device
// (kFirstPassCtas CTAs of kWarpsPerCta warps per SM), cached per device.
int64_t warp_slots() {
  static int64_t slots[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152 * kFirstPassCtas * kWarpsPerCta;
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
  // units start at multiples of 16 rows past y_begin; the top-border
  // replication of the block logic needs every start at row 0 or >= 19
  if (v.y_begin != 0 && v.y_begin < 19) return cudaErrorInvalidValue;
  const int rm_class = strip_class(kp);
  const int uw = strip_width(kp.source == 1, rm_class);
  const int64_t units_x = (v.width + uw - 1) / uw;
  const int uh = unit_height(v.y_end - v.y_begin, units_x, kp);
  const int64_t units_y = (v.y_end - v.y_begin + uh - 1) / uh;
  const int64_t units = units_x * units_y;
  if (units <= 0) return cudaSuccess;
  const int64_t blocks = (units + kWarpsPerCta - 1) / kWarpsPerCta;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (rm_class == kWideRm) return launch_wide(v, kp, s, blocks, units_x, units, uh);
  if (rm_class == kXWideRm) return launch_xwide(v, kp, s, blocks, units_x, units, uh);
  if (rm_class == kCompactRm) return launch_compact(v, kp, s, blocks, units_x, units, uh);
  return v.elem == 1 ? launch_t<uint8_t, kNarrowRm>(v, kp, s, blocks, units_x, units, uh)
                     : launch_t<uint16_t, kNarrowRm>(v, kp, s, blocks, units_x, units, uh);
}

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_stream)
}  // namespace fx
