// fx_api.cpp -- host side of the C ABI: parameters, masks, validation, fx_extract.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "fx_internal.h"

namespace fx {

namespace {

constexpr double kPi = 3.14159265358979323846;

double round_half_away(double v) { return v >= 0.0 ? std::floor(v + 0.5) : -std::floor(-v + 0.5); }

// s > T  <=>  D > floor(T^2 * Lambda * (Lambda - 1))  for integer D >= 0.
int64_t sd_threshold(double T, double lambda) {
  if (T < 0.0) return -1;
  double thr = ((T * T) * lambda) * (lambda - 1.0);
  double fl = std::floor(thr);
  if (!(fl < 9.0e18)) return INT64_MAX;
  return static_cast<int64_t>(fl);
}

// max - min > T  <=>  max - min > floor(T)  for integer max - min >= 0.
int32_t contrast_threshold(double T) {
  if (T < 0.0) return -1;
  double fl = std::floor(T);
  if (!(fl < 2147483647.0)) return INT32_MAX;
  return static_cast<int32_t>(fl);
}

// Eq. 1 (Sec. 3.1) sampled on x, y in {-2..2}, minus its mean; big = max |g|.
bool centred_eq1(double sigma, double g[25], double *big) {
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return false;
  const double s2 = sigma * sigma;
  const double k = -1.0 / (kPi * s2 * s2);
  double total = 0.0;
  for (int i = 0; i < 25; ++i) {
    const double dx = i % 5 - 2, dy = i / 5 - 2;
    const double t = (dx * dx + dy * dy) / (2.0 * s2);
    g[i] = k * (1.0 - t) * std::exp(-t);
    total += g[i];
  }
  const double mean = total / 25.0;
  *big = 0.0;
  for (int i = 0; i < 25; ++i) {
    g[i] -= mean;
    *big = std::fmax(*big, std::fabs(g[i]));
  }
  return *big > 0.0 && std::isfinite(*big);
}

// Largest float <= t (t itself when it is a float).
float float_at_or_below(double t) {
  float f = static_cast<float>(t);
  if (static_cast<double>(f) > t) f = std::nextafter(f, -INFINITY);
  return f;
}

// Ring index (squared radius 0, 1, 2, 4, 5, 8 -> 0..5) of tap i of a 5x5 mask.
int ring_of(int i) {
  const int dx = i % 5 - 2, dy = i / 5 - 2, r2 = dx * dx + dy * dy;
  return r2 == 0 ? 0 : r2 == 1 ? 1 : r2 == 2 ? 2 : r2 == 4 ? 3 : r2 == 5 ? 4 : 5;
}

}  // namespace

fx_status make_kparams(const fx_params *p, int32_t maxval, KParams *kp) {
  if (!p || !kp || p->struct_size != sizeof(fx_params)) return FX_ERR_INVALID_ARG;
  std::memset(kp, 0, sizeof(*kp));
  const double *dv[] = {&p->sigma[0], &p->sigma[1], &p->t_zc[0], &p->t_zc[1], &p->t_sd5[0],
                        &p->t_sd5[1], &p->t_sdmax[0], &p->t_sdmax[1], &p->t_sd3[0], &p->t_sd3[1]};
  for (const double *d : dv)
    if (std::isnan(*d)) return FX_ERR_INVALID_ARG;
  if (p->stddev_source != 0 && p->stddev_source != 1) return FX_ERR_INVALID_ARG;
  if (p->log_mode != FX_LOG_INT && p->log_mode != FX_LOG_FP32) return FX_ERR_INVALID_ARG;
  kp->source = p->stddev_source;
  kp->f32log = p->log_mode == FX_LOG_FP32;
  for (int i = 0; i < FX_MAX_HMF_LEVELS; ++i) {
    int k = p->hmf[i];
    if (k == 0) break;
    if (k != 3 && k != 5 && k != 7) return FX_ERR_INVALID_ARG;
    kp->hmf[kp->nhmf++] = k;
    kp->r_m += k / 2;
  }
  kp->r_in = kp->r_m + (kp->source == 1 ? 2 : 0) + 1 + 2;
  int64_t splus = 0;
  for (int f = 0; f < 2; ++f) {
    fx_status st = fx_log_mask(p->sigma[f], p->mask_q, kp->w[f]);
    if (st != FX_OK) return st;
    static const int rx[6] = {0, 1, 1, 2, 2, 2}, ry[6] = {0, 0, 1, 0, 1, 2};
    for (int c = 0; c < 6; ++c) {
      kp->ring[f][c] = kp->w[f][(ry[c] + 2) * 5 + rx[c] + 2];
      kp->ringf[f][c] = static_cast<float>(kp->ring[f][c]);
    }
    // the construction keeps Eq. 1's radial symmetry; the ring form relies on it
    int64_t pos = 0;
    for (int i = 0; i < 25; ++i) {
      if (kp->w[f][i] != kp->ring[f][ring_of(i)]) return FX_ERR_UNSUPPORTED;
      if (kp->w[f][i] > 0) pos += kp->w[f][i];
    }
    if (pos > splus) splus = pos;
    if (kp->f32log) {  // FP32-LoG mode: the ring weights are the non-integer mask's
      float wf[25];
      st = fx_log_mask_fp32(p->sigma[f], p->mask_q, wf);
      if (st != FX_OK) return st;
      for (int c = 0; c < 6; ++c) kp->ringf[f][c] = wf[(ry[c] + 2) * 5 + rx[c] + 2];
      for (int i = 0; i < 25; ++i)
        if (wf[i] != kp->ringf[f][ring_of(i)]) return FX_ERR_UNSUPPORTED;
      kp->tzf[f] = float_at_or_below(p->t_zc[f]);
    }
    kp->tzc[f] = contrast_threshold(p->t_zc[f]);
    kp->tsd5[f] = sd_threshold(p->t_sd5[f], 25.0);
    kp->tsdmax[f] = sd_threshold(p->t_sdmax[f], 25.0);
    kp->tsd3[f] = sd_threshold(p->t_sd3[f], 9.0);
  }
  kp->splus = splus;
  if (kp->f32log) {
    // FP32 responses need no range condition; the FP32 pass keeps 32-bit
    // standard-deviation sums for values <= 4095 and the wide pass takes the rest.
    kp->fbound = 4095;
  } else {
    // |L| <= maxval * splus for every partial sum; the contrast needs twice that.
    if (2 * static_cast<int64_t>(maxval) * splus >= INT32_MAX) return FX_ERR_RANGE;
    // FP32-exact path: partial sums of L below 2^24 and D below 2^32 (values <= 4095).
    int64_t fb = splus > 0 ? ((1LL << 24) - 1) / splus : 4095;
    if (fb > 4095) fb = 4095;
    kp->fbound = static_cast<int32_t>(fb);
  }
  auto tt = [](int64_t t) -> uint32_t {  // D > t  <=>  D >= t + 1 (D < 2^32)
    if (t < 0) return 0u;
    if (t >= 0xFFFFFFFFLL) return 0xFFFFFFFFu;
    return static_cast<uint32_t>(t + 1);
  };
  for (int f = 0; f < 2; ++f) {
    if (kp->f32log) {
      // fl(max - min) - tzc1f < 0  <=>  fl(max - min) <= tzf  (tzc1f = next float above tzf)
      kp->tzc1f[f] = std::nextafter(kp->tzf[f], INFINITY);
    } else {
      // max - min < 2^25 on the FP32-exact path; tzc + 1 must be exact or out of reach
      const int64_t t1 = static_cast<int64_t>(kp->tzc[f]) + 1;
      if (t1 <= (1LL << 24)) kp->tzc1f[f] = static_cast<float>(t1);
      else if (t1 >= (1LL << 25)) kp->tzc1f[f] = 33554432.0f;
      else kp->fbound = -1;
    }
    kp->tt5[f] = tt(kp->tsd5[f]);
    kp->ttmax[f] = tt(kp->tsdmax[f]);
    kp->tt3[f] = tt(kp->tsd3[f]);
    kp->ntzc1f[f] = -kp->tzc1f[f];
  }
  // Sign-bit form of the FP32 path's standard-deviation tests (values <= fbound
  // <= 4095: D3 <= 20 * 4095^2 < 2^30, D5 <= 156 * 4095^2 < 2^32).  A 3x3
  // threshold above 2^30 is never reached, so it is clamped there; a 5x5
  // threshold above 2^31 is reached only by D5 above 2^31, so such
  // thresholds lower fbound to 3710 (156 * 3710^2 < 2^31) and are clamped too.
  kp->one = 1u;
  for (int f = 0; f < 2; ++f) {
    if (kp->tt3[f] > (1u << 30)) kp->tt3[f] = 1u << 30;
    if (kp->tt5[f] > (1u << 31) || kp->ttmax[f] > (1u << 31)) {
      if (kp->fbound > 3710) kp->fbound = 3710;
      if (kp->tt5[f] > (1u << 31)) kp->tt5[f] = 1u << 31;
      if (kp->ttmax[f] > (1u << 31)) kp->ttmax[f] = 1u << 31;
    }
    kp->ntt3[f] = 0u - kp->tt3[f];
    kp->ntt5[f] = 0u - kp->tt5[f];
    kp->nttmax[f] = 0u - kp->ttmax[f];
  }
  kp->sd_same = kp->tsd5[0] == kp->tsd5[1] && kp->tsdmax[0] == kp->tsdmax[1] && kp->tsd3[0] == kp->tsd3[1];
  // crossing-map source: the counts n in [0, Lambda] with n (Lambda - n) > t form
  // an interval (the product is concave in n); encode its bounds bit by bit
  auto interval = [](int64_t t, int lambda, int bits, uint32_t *sel) {
    int lo = (1 << bits) - 1, hi = 0;
    for (int n = lambda; n >= 0; --n)
      if (static_cast<int64_t>(n) * (lambda - n) > t) lo = n;
    for (int n = 0; n <= lambda; ++n)
      if (static_cast<int64_t>(n) * (lambda - n) > t) hi = n;
    for (int i = 0; i < bits; ++i) {
      sel[i] = (lo >> i) & 1 ? 0xFFFFFFFFu : 0u;
      sel[bits + i] = (hi >> i) & 1 ? 0xFFFFFFFFu : 0u;
    }
  };
  for (int f = 0; f < 2; ++f) {
    interval(kp->tsd5[f], 25, 5, kp->zsel[f]);
    interval(kp->tsdmax[f], 25, 5, kp->zsel[f] + 10);
    interval(kp->tsd3[f], 9, 4, kp->zsel[f] + 20);
  }
  return FX_OK;
}

fx_status check_image(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                      int32_t dtype, const uint8_t *out, int64_t out_pitch) {
  if (!img || !out) return FX_ERR_INVALID_ARG;
  if (dtype != FX_U8 && dtype != FX_U16) return FX_ERR_INVALID_ARG;
  const int64_t elem = dtype == FX_U8 ? 1 : 2;
  if (width < 1 || height < 1 || width > (1LL << 30) || height > (1LL << 30)) return FX_ERR_INVALID_ARG;
  if (pitch_bytes < width * elem || pitch_bytes % elem != 0 || pitch_bytes > 0xFFFFFFFFLL) return FX_ERR_INVALID_ARG;
  if (out_pitch < width || out_pitch > 0xFFFFFFFFLL) return FX_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(img) % elem != 0) return FX_ERR_INVALID_ARG;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(img);
  const uintptr_t a1 = a0 + (height - 1) * pitch_bytes + width * elem;
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(out);
  const uintptr_t b1 = b0 + (height - 1) * out_pitch + width;
  if (a0 < b1 && b0 < a1) return FX_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FX_ERR_CUDA;
  for (const void *ptr : {img, static_cast<const void *>(out)}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return FX_ERR_INVALID_ARG;
    }
    if (at.type == cudaMemoryTypeManaged) continue;
    if (at.type != cudaMemoryTypeDevice || at.device != dev) return FX_ERR_INVALID_ARG;
  }
  return FX_OK;
}

cudaError_t launch_extract(const ImageView &v, const KParams &kp, cudaStream_t s) {
  if (fast_path_supported(kp)) return launch_fast(v, kp, s);
  return launch_tile_general(v, kp, s);
}

}  // namespace fx

using namespace fx;

extern "C" {

void fx_params_default(fx_params *p, fx_dtype dtype, int32_t bits) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(fx_params);
  if (bits <= 0) bits = dtype == FX_U8 ? 8 : 12;
  const double s = bits > 8 ? std::ldexp(1.0, bits - 8) : 1.0;
  p->sigma[0] = 0.5;
  p->sigma[1] = 20.0;
  p->mask_q = 512;
  p->t_zc[0] = 4248.0 * s;
  p->t_zc[1] = 15360.0 * s;
  for (int f = 0; f < 2; ++f) {
    p->t_sd5[f] = 6.0 * s;
    p->t_sd3[f] = 6.0 * s;
    p->t_sdmax[f] = 24.0 * s;
  }
  p->stddev_source = 0;
  p->hmf[0] = 5;
  p->bits = bits;
  p->out_pitch = 0;
}

// Eq. 1 sampled on the 5x5 grid; mean removed; scaled so that max |w| = Q;
// rounded half away from zero; centre tap reset to make the mask zero-sum.
fx_status fx_log_mask(double sigma, int32_t mask_q, int32_t w[25]) {
  double g[25], big = 0.0;
  if (!w || mask_q < 1 || !centred_eq1(sigma, g, &big)) return FX_ERR_INVALID_ARG;
  int64_t rest = 0;
  for (int i = 0; i < 25; ++i) {
    const double r = round_half_away(static_cast<double>(mask_q) * g[i] / big);
    if (!(std::fabs(r) < 1e9)) return FX_ERR_RANGE;
    w[i] = static_cast<int32_t>(r);
    if (i != 12) rest += w[i];
  }
  if (rest > INT32_MAX || rest < -INT32_MAX) return FX_ERR_RANGE;
  w[12] = static_cast<int32_t>(-rest);
  return FX_OK;
}

// The same samples on the grid 2^(e-23), 2^e the smallest power of two >= Q:
// every weight then has at most 24 significant bits (exact in FP32) and the
// centre, minus the exact sum of the other 24, keeps the mask zero-sum.
fx_status fx_log_mask_fp32(double sigma, int32_t mask_q, float w[25]) {
  double g[25], big = 0.0;
  if (!w || mask_q < 1 || !centred_eq1(sigma, g, &big)) return FX_ERR_INVALID_ARG;
  if (mask_q > (1 << 20)) return FX_ERR_RANGE;
  int e = 0;
  while ((int64_t{1} << e) < mask_q) ++e;
  const double grid = std::ldexp(1.0, e - 23), lim = std::ldexp(1.0, e + 1);
  double v[25], rest = 0.0;
  for (int i = 0; i < 25; ++i) {
    v[i] = round_half_away(static_cast<double>(mask_q) * g[i] / big / grid) * grid;
    if (i != 12) rest += v[i];  // exact: multiples of grid below 2^(e+6)
  }
  v[12] = -rest;
  for (int i = 0; i < 25; ++i) {
    if (!(std::fabs(v[i]) < lim)) return FX_ERR_RANGE;
    w[i] = static_cast<float>(v[i]);
  }
  return FX_OK;
}

fx_status fx_extract(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                     fx_dtype dtype, const fx_params *params, uint8_t *out_mask, void *stream) {
  NvtxRange range("fx_extract");
  fx_params def;
  if (!params) {
    fx_params_default(&def, dtype, 0);
    params = &def;
  }
  if (params->struct_size != sizeof(fx_params)) return FX_ERR_INVALID_ARG;
  const int64_t out_pitch = params->out_pitch ? params->out_pitch : width;
  fx_status st = check_image(img, width, height, pitch_bytes, dtype, out_mask, out_pitch);
  if (st != FX_OK) return st;
  KParams kp;
  st = make_kparams(params, dtype == FX_U8 ? 255 : 65535, &kp);
  if (st != FX_OK) return st;
  ImageView v{img, width, height, pitch_bytes, 0, dtype == FX_U8 ? 1 : 2, out_mask, out_pitch, 0, height, height};
  return launch_extract(v, kp, static_cast<cudaStream_t>(stream)) == cudaSuccess ? FX_OK : FX_ERR_CUDA;
}

const char *fx_status_string(fx_status s) {
  switch (s) {
    case FX_OK: return "FX_OK";
    case FX_ERR_INVALID_ARG: return "FX_ERR_INVALID_ARG";
    case FX_ERR_UNSUPPORTED: return "FX_ERR_UNSUPPORTED";
    case FX_ERR_RANGE: return "FX_ERR_RANGE";
    case FX_ERR_CUDA: return "FX_ERR_CUDA";
    case FX_ERR_NOMEM: return "FX_ERR_NOMEM";
    case FX_ERR_BUDGET: return "FX_ERR_BUDGET";
    case FX_ERR_TIMEOUT: return "FX_ERR_TIMEOUT";
  }
  return "FX_ERR_UNKNOWN";
}

const char *fx_version(void) { return "fx 1.0 sm_103a"; }

}  // extern "C"

namespace fx {
bool checked_build() {
#ifdef FX_CHECKED
  return true;
#else
  return false;
#endif
}
}  // namespace fx

namespace fx {
// check counters of the batched path's compact and wide kernels (fx_plan_compact.cu, fx_plan_wide.cu)
unsigned long long checked_count_plan_compact(bool reset);
unsigned long long checked_count_plan_wide(bool reset);
unsigned long long checked_count_plan_xwide(bool reset);
}  // namespace fx

extern "C" fx_status fx_checked_violations(uint64_t *count, int32_t reset) {
  if (!count) return FX_ERR_INVALID_ARG;
  *count = 0;
  if (!fx::checked_build()) return FX_ERR_UNSUPPORTED;
  if (cudaDeviceSynchronize() != cudaSuccess) return FX_ERR_CUDA;
  unsigned long long (*const readers[])(bool) = {fx::checked_count_stream, fx::checked_count_stream_wide,
                                                  fx::checked_count_stream_compact,
                                                  fx::checked_count_tile, fx::checked_count_plan, fx::checked_count_plan_compact, fx::checked_count_plan_wide,
                                                  fx::checked_count_plan_xwide, fx::checked_count_stream_xwide,
                                                  fx::checked_count_noalloc, fx::checked_count_hmf};
  uint64_t total = 0;
  for (auto r : readers) {
    const unsigned long long c = r(reset != 0);
    if (c == ~0ULL) return FX_ERR_CUDA;
    total += c;
  }
  *count = total;
  return FX_OK;
}
