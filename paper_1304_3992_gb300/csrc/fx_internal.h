// fx_internal.h -- types shared by the host side of libfx and its kernels.
// Kernels compiled at run time (fx_jit.cpp) see the types only: the host
// declarations are left out under __CUDACC_RTC__.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#endif

#include "../../include/fx.h"

namespace fx {

// Per-call constants of the method, derived on the host from fx_params.
struct KParams {
  // Integer LoG masks (Eq. 1 reading), row-major 5x5, and their 6 ring values
  // for squared radii 0, 1, 2, 4, 5, 8 (the masks are radial, hence D4-symmetric).
  int32_t w[2][25];
  int32_t ring[2][6];
  float ringf[2][6];
  // Contrast test max - min > t_zc  <=>  max - min > tzc (integers).
  int32_t tzc[2];
  // Standard-deviation tests s > T  <=>  D > t with D = Lambda*sum(a^2) - (sum a)^2
  // and t = floor(T^2 Lambda (Lambda-1)) (-1 when T < 0, i.e. always true).
  int64_t tsd5[2], tsdmax[2], tsd3[2];
  int32_t source;  // 0 = image, 1 = binary zero-crossing map
  int32_t nhmf;    // number of hybrid-median passes
  int32_t hmf[FX_MAX_HMF_LEVELS];
  int32_t r_m;     // total radius of the median passes
  int32_t r_in;    // input radius of one output pixel
  // Largest sum of positive taps over both masks; bounds |L| <= maxval * splus.
  int64_t splus;
  // --- streaming fast path (fx_stream.cuh) ---
  // Largest input value the first (FP32) pass handles: with the integer masks
  // every LoG partial sum below 2^24, D below 2^32 and t_zc + 1 representable;
  // in the FP32-LoG mode D below 2^32 (4095).  -1 = never (all strips redone).
  int32_t fbound;
  // FP32 contrast test: (max - min) - tzc1f < 0  <=>  max - min <= t_zc.
  float tzc1f[2];
  // 32-bit standard-deviation tests for the FP32 path: s > T  <=>  D >= tt.
  uint32_t tt5[2], ttmax[2], tt3[2];
  // The same tests as sign bits: with r = D - tt (mod 2^32), D3 < 2^31 and
  // tt3 <= 2^30, D3 < tt3 <=> r3 < 0; D5 < 2^32 and tt5, ttmax <= 2^31, so
  // D5 < tt <=> (D5 < 2^31 and r < 0).  ntt* = -tt* (mod 2^32); one = 1 (an
  // opaque multiplier, so the subtraction stays a multiply-add).
  uint32_t ntt5[2], nttmax[2], ntt3[2], one;
  // -tzc1f, the contrast threshold of the FP32 path added to max - min
  float ntzc1f[2];
  int32_t sd_same;   // both branches use the same standard-deviation thresholds
  // FP32-LoG mode (fx_params.log_mode): ringf holds the non-integer mask's ring
  // weights and L is evaluated in FP32 from d_c = R_c - n_c I(p); the contrast
  // test is fl(max - min) > tzf (t_zc rounded down to FP32).
  int32_t f32log;
  float tzf[2];
  // Crossing-map source (source 1): with n crossings in a window of Lambda
  // pixels D = n (Lambda - n), so each test D > t holds for n in an interval.
  // Per branch, bit masks (all ones / zero) of the interval bounds, LSB first:
  // [0..4] lo and [5..9] hi of the 5x5 test, [10..19] of the 5x5 test against
  // t_sdmax, [20..23] lo and [24..27] hi of the 3x3 test.  An empty interval
  // has lo above every count.
  uint32_t zsel[2][28];
};

#ifndef __CUDACC_RTC__
// NVTX range over a host-side scope (launches, copies, pipeline stages); the
// ranges cost nothing unless a profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
#endif

// Derive KParams from fx_params for images whose values are <= maxval.
fx_status make_kparams(const fx_params *p, int32_t maxval, KParams *kp);

// Validation shared by fx_extract and the descriptors of fx_extract_batch.
fx_status check_image(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                      int32_t dtype, const uint8_t *out, int64_t out_pitch);

// Launchers (fx_tile.cu, fx_stream.cu).  Row window: output rows [y_begin, y_end)
// of an image of height `height`; `img` points at image row `row0` (the buffer
// holds rows [row0, ...)), `out` at output row y_begin.
struct ImageView {
  const void *img;
  int64_t width, height, pitch;  // pitch in bytes
  int64_t row0;                  // image row held at img
  int32_t elem;                  // 1 or 2
  uint8_t *out;
  int64_t out_pitch;
  int64_t y_begin, y_end;
  int64_t row_lim;               // rows [row0, row_lim) are present in the buffer
};

#ifndef __CUDACC_RTC__
cudaError_t launch_tile_general(const ImageView &v, const KParams &kp, cudaStream_t s);

// Range-check failures counted by the kernels of each translation unit (the
// FX_CHECKED build; 0 otherwise, ~0 when the counter cannot be read).
unsigned long long checked_count_stream(bool reset);
unsigned long long checked_count_stream_wide(bool reset);
unsigned long long checked_count_stream_compact(bool reset);
unsigned long long checked_count_stream_xwide(bool reset);
unsigned long long checked_count_tile(bool reset);
unsigned long long checked_count_plan(bool reset);
unsigned long long checked_count_noalloc(bool reset);
unsigned long long checked_count_hmf(bool reset);
bool checked_build();
bool fast_path_supported(const KParams &kp);  // the streaming kernels (compact, narrow, wide or extra-wide strips)
int strip_class(const KParams &kp);           // the smallest strip class that serves kp (its median radius sum)
cudaError_t launch_compact(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                           int64_t units, int uh);
cudaError_t launch_wide(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                        int64_t units, int uh);
cudaError_t launch_xwide(const ImageView &v, const KParams &kp, cudaStream_t s, int64_t blocks, int64_t units_x,
                         int64_t units, int uh);
bool pair_loads_ok(const ImageView &v);
bool pair_loads_ok(const void *img, int64_t width, int64_t pitch, int64_t elem);
cudaError_t launch_fast(const ImageView &v, const KParams &kp, cudaStream_t s);
cudaError_t launch_extract(const ImageView &v, const KParams &kp, cudaStream_t s);
// The first-pass kernel compiled at run time for kp's masks and contrast
// thresholds (fx_specialize) for this pixel size, load path and strip class on
// the current device, or nullptr (fx_jit.cpp).
const void *specialized_kernel(const KParams &kp, int elem, bool pair, int rm_class);
#endif

}  // namespace fx
