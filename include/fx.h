/*
 * fx.h -- C ABI of the GB300 feature-extraction library (libfx.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the data-parallel
 * feature-extraction path of "GPU Accelerated Automated Feature Extraction
 * from Satellite Images" (arXiv 1304.3992): for every pixel of a single-band
 * uint8/uint16 image
 *   1. two 5x5 Laplacian-of-Gaussian responses L1, L2 (Sec. 3.1, Eq. 1,
 *      sigma 0.5 and 20 per Sec. 4.1);
 *   2. zero crossings of each response among the 4 neighbours, kept when the
 *      positive maximum minus the negative minimum exceeds a threshold
 *      (Sec. 3.2, Sec. 4);
 *   3. the local standard-deviation test (Eq. 2): 5x5 window, re-computed on
 *      the 3x3 window above a maximum threshold (Sec. 4.1);
 *   4. OR-combination of the two extracted maps (Sec. 4.1);
 *   5. an optional hybrid median filter (Sec. 3.4), optionally repeated with
 *      several window sizes (Sec. 4, Sec. 4.2).
 * The output is a binary mask, one uint8 (0 or 1) per pixel.
 *
 * Readings where the paper is silent (the masks are the zero-sum integer
 * rounding of Eq. 1 scaled to max |w| = mask_q; every stage extends past the
 * image border by replication; zero-crossing ties go to the negative pixel;
 * s > T is decided exactly as Lambda*sum(a^2) - (sum a)^2 > T^2 Lambda
 * (Lambda-1); the combination is OR) are fixed here and documented per field.
 *
 * Conventions for every entry point:
 *   - All image and mask pointers are DEVICE pointers unless the name says
 *     _host.  The caller owns them; the library never frees them and keeps no
 *     reference after the call returns.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and runs asynchronously; the returned status reports host-side
 *     validation and launch errors only.
 *   - On any error nothing is launched and no output byte is written.
 *   - No call throws; no call prints.
 *   - In the default integer-mask mode results are bit-identical to the
 *     definition above for every input value (exact integer / FP32-exact
 *     arithmetic).  The optional FP32-LoG mode (fx_params.log_mode) uses
 *     non-integer masks and FP32 responses; its results differ from the exact
 *     definition only where a decision is within rounding of its threshold.
 */
#ifndef FX_H
#define FX_H

#ifndef __CUDACC_RTC__ /* kernels compiled at run time bring their own fixed-width types */
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FX_OK = 0,
  FX_ERR_INVALID_ARG = 1, /* null pointer, bad size/pitch/alignment/dtype, NaN parameter */
  FX_ERR_UNSUPPORTED = 2, /* valid request outside what the library implements */
  FX_ERR_RANGE = 3,       /* parameters whose exact evaluation would overflow 32-bit sums */
  FX_ERR_CUDA = 4,        /* a CUDA runtime call or a launch failed */
  FX_ERR_NOMEM = 5,       /* a device or pinned-host allocation failed */
  FX_ERR_BUDGET = 6,      /* request larger than a configured memory budget */
  FX_ERR_TIMEOUT = 7      /* a bounded device-side wait gave up */
} fx_status;

typedef enum { FX_U8 = 1, FX_U16 = 2 } fx_dtype;

#define FX_MAX_HMF_LEVELS 4

/* LoG evaluation modes (fx_params.log_mode). */
typedef enum {
  FX_LOG_INT = 0, /* integer masks, exact responses (default) */
  FX_LOG_FP32 = 1 /* non-integer masks from Eq. 1, FP32 responses */
} fx_log_mode;

typedef struct {
  /* sizeof(fx_params); set by fx_params_default, checked by every call. */
  uint32_t struct_size;
  /* Gaussian sigma of the two LoG masks (Eq. 1; Sec. 4.1 uses 0.5 and 20). */
  double sigma[2];
  /* Integer mask scale Q: the mean-removed Eq. 1 samples are scaled to
   * max |w| = Q, rounded half away from zero, and the centre tap is reset to
   * minus the sum of the other 24 (zero-sum).  Default 512. */
  int32_t mask_q;
  /* Zero-crossing contrast thresholds per branch, in response units:
   * keep a crossing when max - min of L over it and its 4 neighbours > t_zc. */
  double t_zc[2];
  /* Standard-deviation thresholds per branch, in image units (Eq. 2):
   * S = (s5 > t_sdmax) ? (s3 > t_sd3) : (s5 > t_sd5).  A negative threshold
   * always passes. */
  double t_sd5[2], t_sdmax[2], t_sd3[2];
  /* 0 = the standard deviation is taken over the image (default); 1 = over
   * the binary zero-crossing map of the same branch (Sec. 4.1 literal). */
  int32_t stddev_source;
  /* Hybrid-median windows applied in order (3, 5 or 7; 0 ends the list;
   * Sec. 3.4 leaves the size to the application, Sec. 4.2 repeats the filter
   * with several sizes).  Default {5, 0, 0, 0}; all zero switches the filter
   * off.  fx_extract runs lists whose radii (window / 2) add up to at most 11
   * in its fused streaming kernel, longer ones in the general tile kernel. */
  int32_t hmf[FX_MAX_HMF_LEVELS];
  /* Nominal radiometric depth used only to scale the default thresholds
   * (value scale 2^(bits-8)); it never restricts the input values. */
  int32_t bits;
  /* Row pitch of out_mask in bytes for fx_extract; 0 = width. */
  int64_t out_pitch;
  /* FX_LOG_INT (default) or FX_LOG_FP32.  In FX_LOG_FP32 the masks are the
   * mean-removed Eq. 1 samples scaled to max |w| = mask_q and rounded half
   * away from zero to multiples of g = 2^(e - 23), 2^e the smallest power of
   * two >= mask_q (g = 2^-14 for 512), with the centre reset to minus the sum
   * of the other 24 (zero-sum and exact in FP32); see fx_log_mask_fp32.  Each
   * response is evaluated in FP32 from exact ring sums R_c of the radial
   * mask (squared radii c = 1, 2, 4, 5, 8, n_c pixels each) as
   *   L = w1 d1 (+) w2 d2 (+) w4 d4 (+) w5 d5 (+) w8 d8,  d_c = R_c - n_c I(p),
   * left to right with one rounding per product-add (fused multiply-add), and
   * -0 read as +0.  The contrast test is fl(max - min) > t_zc with t_zc
   * rounded down to FP32; the standard-deviation test stays exact.  Zero
   * crossings and contrast then differ from the exact responses only where
   * |L|, |L(p) + L(q)| or |max - min - t_zc| is within FP32 rounding of 0. */
  int32_t log_mode;
  int32_t reserved;
} fx_params;

/*
 * Fill *p with the defaults: sigma {0.5, 20}, mask_q 512, hmf {5}, image
 * stddev source, and thresholds for a 12-DN step on 8-bit data times the
 * value scale s = 2^(bits-8): t_zc = {4248 s, 15360 s}, t_sd5 = t_sd3 = 6 s,
 * t_sdmax = 24 s.  bits = 0 selects 8 for FX_U8 and 12 for FX_U16 (the
 * 12-bit radiometry of the paper's AWiFS scenes, Sec. 6).  p may not be NULL.
 */
void fx_params_default(fx_params *p, fx_dtype dtype, int32_t bits);

/*
 * The integer mask of one branch (reading of Eq. 1 above) into w[25]
 * (row-major, w[(dy+2)*5 + dx+2]).  Returns FX_ERR_INVALID_ARG for sigma <= 0,
 * mask_q < 1 or non-finite values.
 */
fx_status fx_log_mask(double sigma, int32_t mask_q, int32_t w[25]);

/*
 * The FX_LOG_FP32 mask of one branch (see fx_params.log_mode) into w[25]
 * (row-major).  Every weight is a multiple of 2^(e - 23) with |w| < 2^(e+1),
 * so it is exact in FP32, and the 25 weights sum to exactly zero.  Host only.
 * Returns FX_ERR_INVALID_ARG for sigma <= 0, mask_q < 1 or non-finite values,
 * FX_ERR_RANGE when mask_q > 2^20.
 */
fx_status fx_log_mask_fp32(double sigma, int32_t mask_q, float w[25]);

/*
 * One image, stateless (Sec. 4.1 flow, one fused kernel launch).
 *   img          device pointer to row 0; aligned to the element size
 *   width,height pixels, both >= 1
 *   pitch_bytes  distance between image rows, >= width*elem, multiple of elem,
 *                below 2^32
 *   dtype        FX_U8 or FX_U16
 *   params       NULL = fx_params_default(dtype, 0)
 *   out_mask     device pointer, height rows of params->out_pitch (or width)
 *                bytes, out_pitch below 2^32; must not overlap the image
 * Errors: FX_ERR_INVALID_ARG, FX_ERR_RANGE, FX_ERR_UNSUPPORTED, FX_ERR_CUDA.
 * Thread-safe; allocates nothing.
 */
fx_status fx_extract(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                     fx_dtype dtype, const fx_params *params, uint8_t *out_mask, void *stream);

/* ------------------------------------------------------------------ plans */

typedef struct fx_plan fx_plan;

/*
 * A plan fixes the parameters and owns the device workspace of the batched
 * path: descriptor table, tile-queue counter, device status word, cached CUDA
 * graph and the tuned tile configuration.  One host thread uses a plan at a
 * time.  max_images bounds fx_extract_batch's n (>= 1).  device is the CUDA
 * device ordinal the workspace lives on.
 * Errors: FX_ERR_INVALID_ARG, FX_ERR_RANGE, FX_ERR_NOMEM, FX_ERR_CUDA.
 */
fx_status fx_plan_create(fx_plan **plan, const fx_params *params, int32_t max_images,
                         int32_t device);

/* Releases the plan's workspace after waiting for its outstanding work. */
fx_status fx_plan_destroy(fx_plan *plan);

typedef struct {
  const void *img;     /* device pointer to row 0 of the image */
  int64_t width, height, pitch_bytes;
  int32_t dtype;       /* fx_dtype */
  int32_t reserved;
  uint8_t *out_mask;   /* device pointer */
  int64_t out_pitch;   /* bytes; 0 = width */
} fx_image_desc;

/*
 * Many images of uneven sizes and mixed dtypes in ONE replay of a CUDA graph:
 * persistent kernels pop work units from a tile queue (one kernel per load
 * path and pixel type on the streaming path, then the redo pass), the batched
 * form of Sec. 6.2.2's one-thread-per-pixel mapping.  Median lists whose radii
 * add up to at most 11 run on the streaming strips of fx_extract (compact,
 * narrow, wide or extra wide), longer lists on the general tile kernel.
 * Each image's mask is byte-identical to fx_extract's.  descs is a HOST array
 * of n descriptors, validated like fx_extract's arguments; the table is
 * copied before the call returns.
 * Output masks must not overlap each other or any input.
 * The plan holds two descriptor tables and two sets of queue counters and
 * alternates between them, so two calls on one plan may run at the same time
 * (for example on two streams); a third call waits on the host until the
 * first one's replay has finished.  Calls on one plan must come from one host
 * thread at a time.  The plan's device is made current for the call and the
 * caller's current device is restored before it returns.
 * Errors: FX_ERR_INVALID_ARG (n < 1, n > max_images, bad descriptor),
 * FX_ERR_CUDA.
 */
fx_status fx_extract_batch(fx_plan *plan, const fx_image_desc *descs, int32_t n, void *stream);

/*
 * Work-unit shape of the batched kernel and its CTAs per SM.  A unit is a
 * strip of tile_w output columns by tile_h output rows walked by one warp;
 * tile_w must be the strip width of the plan's streaming strips: 56 with no
 * median or one window-3 median, 52 while the median radii add up to at most
 * 3 (the default window 5 included), 44 up to 7, 36 up to 11; 4 fewer when
 * the standard deviation is taken over the crossing map.  tile_h is a multiple
 * of 16 in [16, 8192], or 0; ctas_per_sm is in 1..32 (one warp per CTA on
 * the streaming kernels, 256 threads on the general kernel).
 * A new plan picks the unit height for each batch itself (multiples of 16 up
 * to 1024, from the batch's unit count against the resident warps; 12 CTAs
 * per SM) until one of the two calls below fixes another shape.
 * fx_plan_autotune times the automatic height and the heights
 * {256, 512, 768, 1024} x three CTAs-per-SM counts (12, 10 and 8 on the
 * streaming kernels; 1 .. 8 as the general kernel's occupancy allows) on the
 * given images (their outputs are overwritten) and keeps the fastest;
 * fx_plan_set_tile forces one.  In both calls tile_h 0 stands for the
 * automatic height (picked per batch for the given CTAs per SM).  Plans whose
 * parameters need the general kernel (median windows whose radii add up to
 * more than 11) use its fixed 64 x 32 tile; for them
 * only ctas_per_sm takes effect.
 * Errors: FX_ERR_INVALID_ARG (shape or count out of range), FX_ERR_CUDA.
 */
fx_status fx_plan_autotune(fx_plan *plan, const fx_image_desc *descs, int32_t n, void *stream,
                           int32_t *tile_w, int32_t *tile_h, int32_t *ctas_per_sm);
fx_status fx_plan_set_tile(fx_plan *plan, int32_t tile_w, int32_t tile_h, int32_t ctas_per_sm);

/*
 * Synchronises `stream` and reads the plan's device status word, which the
 * batched kernel sets when a descriptor fails its device-side check or a
 * bounded wait gives up; the word is cleared by the read.
 */
fx_status fx_get_device_status(fx_plan *plan, void *stream);

/*
 * End-to-end call on HOST buffers: copies the image to the device in row
 * chunks of about 64 MiB, extracts, and copies the mask back; the upload of a
 * chunk, the kernel of the previous one and the download of the one before
 * run at the same time on the plan's own streams (three staging slots).  Host
 * buffers should be page-locked for full copy speed.  Synchronous: the mask
 * is in out_mask_host when the call returns.  The plan grows its staging
 * buffers on first use.
 * Errors: as fx_extract, plus FX_ERR_NOMEM.
 */
fx_status fx_extract_host(fx_plan *plan, const void *img_host, int64_t width, int64_t height,
                          int64_t pitch_bytes, fx_dtype dtype, uint8_t *out_mask_host,
                          int64_t out_pitch);

/*
 * fx_extract_host for n images in one call (descs[i].img and .out_mask are
 * HOST pointers here): the row chunks of all images share one copy / kernel /
 * copy pipeline, so uploads of the next image overlap the work on the
 * previous one.  Synchronous; descs is read before the call returns.
 * Errors: as fx_extract_host (n < 1 or a bad descriptor: FX_ERR_INVALID_ARG).
 */
fx_status fx_extract_host_batch(fx_plan *plan, const fx_image_desc *descs, int32_t n);

/*
 * The hybrid median filter of Sec. 3.4 on its own, applied to a uint8/uint16
 * image (grayscale values rather than the binary extraction map): each output
 * pixel is the median of (median of the '+' subgroup, median of the 'x'
 * subgroup, centre), the subgroups being the centre row and column segment
 * and the two diagonals of the window x window neighbourhood; pixels outside
 * the image take the nearest image value.
 *   img, out     device pointers, same dtype; must not overlap
 *   pitch_bytes  input row pitch; out_pitch_bytes output row pitch (0 = packed)
 *   window       3, 5 or 7
 * Errors: FX_ERR_INVALID_ARG, FX_ERR_CUDA.  Allocates nothing.
 */
fx_status fx_hybrid_median(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                           fx_dtype dtype, int32_t window, void *out, int64_t out_pitch_bytes,
                           void *stream);

/*
 * Batched extraction for callers that cannot allocate device memory.  The
 * paper has no counterpart; this entry point exists for deployment: services
 * whose device memory all belongs to another allocator (a framework's caching
 * pool, a fixed arena), real-time loops that forbid cudaMalloc after start-up
 * (it can synchronise the device and fail under fragmentation), and plug-ins
 * handed buffers but no right to allocate.  It does what fx_extract_batch
 * does (same masks, byte for byte) without a plan: the descriptor table
 * travels in the kernel's launch parameters, and its only scratch, the
 * tile-queue counter, sits in a fixed 256-byte array inside the library that
 * every GPU loading libfx.so reserves until process exit.  The call allocates
 * nothing on host or device.
 *   params  NULL = fx_params_default(FX_U16, 0)
 *   descs   HOST array of n descriptors, validated like fx_extract's
 *           arguments; read before the call returns
 *   n       1 .. FX_NOALLOC_MAX_IMAGES; a larger n returns FX_ERR_BUDGET and
 *           launches nothing
 * The first call on a device looks up the scratch array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  Every call on a device shares the one counter, which
 * keeps the last call's value (each call resets it to zero on its stream
 * before its kernel), so calls whose work overlaps on the GPU race: serialise
 * them (one stream, or events).
 * Errors: FX_ERR_INVALID_ARG, FX_ERR_RANGE, FX_ERR_BUDGET, FX_ERR_CUDA.
 */
#define FX_NOALLOC_MAX_IMAGES 128
fx_status fx_extract_batch_noalloc(const fx_params *params, const fx_image_desc *descs, int32_t n,
                                   void *stream);

/*
 * Compiles, at run time on the current device, fx_extract's streaming first
 * pass for this parameter set and dtype with the two LoG masks' ring weights
 * and the contrast thresholds as compile-time constants (NVRTC; a second or
 * two per call, cached for the life of the process); likewise the batched
 * path's group kernels.  Afterwards fx_extract and the host-buffer entry
 * points use these kernels whenever their parameters match, and so do the
 * graphs of plans created afterwards; other calls use the library's
 * precompiled kernels.  The masks are
 * identical either way (the same operations, in the same order).  A tuning
 * aid of this library; the paper has no counterpart.
 * Errors: FX_ERR_INVALID_ARG, FX_ERR_RANGE; FX_ERR_UNSUPPORTED when the
 * parameters do not run on the streaming kernel, the library is the checked
 * build, or run-time compilation is unavailable or fails (then nothing
 * changes); FX_ERR_CUDA.
 */
fx_status fx_specialize(const fx_params *params, fx_dtype dtype);

/*
 * Range-check failures counted by the kernels of the checked build
 * (libfx_checked.so, compiled with FX_CHECKED: every global and shared-memory
 * index of the kernels is checked before use; a failed check is counted and
 * its access skipped, nothing traps).  A debugging aid of this library; the
 * paper has no counterpart.  Synchronises the current device; *count receives
 * the failures counted on it since the last reset, reset != 0 clears them.
 * The normal build returns FX_ERR_UNSUPPORTED with *count = 0.
 */
fx_status fx_checked_violations(uint64_t *count, int32_t reset);

/* Human-readable name of a status code (static storage). */
const char *fx_status_string(fx_status s);

/* Library version, e.g. "fx 1.0 sm_103a". */
const char *fx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FX_H */
