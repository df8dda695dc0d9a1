// fx_stream.cuh -- the streaming fast path (device code).
//
// One warp computes a strip of 52 output columns (48 with the crossing-map
// standard deviation) over a range of output rows, walking down the image one
// row per step.  Lane l owns the two adjacent window columns xs + 2l,
// xs + 2l + 1 of a 64-column window that starts 6 (8) columns left of the
// strip: the halo the stages need (2 LoG + 1 crossing (+ 2 deviation) + up to
// 3 median), rounded up to the even column alignment of the loads.  Two
// columns per lane keep the per-lane state small, so that several warps per
// scheduler hide each other's latencies.
//
// Per step (one input row t; every value stays in registers):
//   - the lane's two pixels of row t + 4 are loaded into a period-4 ring (one
//     aligned pair load, or two single-pixel loads), unconditionally; the
//     replicated border columns are selected when the row is used, and the
//     +-2-column halo comes from the neighbouring lanes by shuffle;
//   - horizontal sums h1 = I(x-1) + I(x+1), h2 = I(x-2) + I(x+2) in FP32, and
//     the 3- and 5-wide sums of squares of the pixels' biased FP32 bits;
//   - for the centre row c = t-2: the six ring sums R0..R8 of the radial
//     masks (squared radii 0, 1, 2, 4, 5, 8), L_f = sum_c w_fc R_c for both
//     masks (Eq. 1, reading R1; FP32-LoG mode: from R_c - n_c I), and the
//     standard-deviation test of Eq. 2 from exact sums (reading R4);
//   - for row c' = t-3 (whose four neighbours are now known): the sign of L,
//     the sign of -L, the signs of the east and south edge sums L(p)+L(q) and
//     the contrast test (Sec. 3.2), each packed as one bit per pixel.
// Bits are packed into 32-bit words covering 16 rows x the lane's 2 columns
// (bit 30 - 2r + j for row r, column j).  Every 16 rows the zero-crossing rule
// (reading R3), the standard deviation over the crossing map (source 1), the
// extraction, the OR of the two maps (Sec. 4.1) and one or two hybrid median
// levels (Sec. 3.4, reading R6) run as bitwise logic on those words, and the
// finished mask rows are stored.  Each 4-row iteration runs a checked body
// (border fix-ups, clamped loads) only where the strip touches a border.
// Single-image launches stop computing steps past the last row any output
// needs (the remaining iterations only shift the bit accumulators); the
// batched kernels, whose units are long, walk the whole block schedule.
//
// Arithmetic is exact with the integer masks: the FP32 path is used while
// every input value is at most KParams::fbound (all LoG partial sums below
// 2^24, Eq. 2's D below 2^32); a strip that meets a larger value is
// recomputed on the integer path (int32 LoG, int64 D).  Borders follow reading
// R2 (every stage replicated): loads clamp, and the L values and the bits of
// every binary stage at rows / columns outside the image are replaced by
// those of the nearest image row / column.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "fx_checked.cuh"
#include "fx_internal.h"

namespace fx {

// Strip classes, by the largest sum of median radii r they serve: compact
// (r <= 1: no median or one window-3 median), narrow (r <= 3), wide (r <= 7)
// and extra wide (r <= 11, e.g. 7, 7, 7).  A 64-column window has 3 + r halo
// columns on each side (2 LoG + 1 crossing + r median), 2 more when the
// standard deviation is taken over the crossing map (its 5x5 window), so a
// strip has 58 - 2r output columns: 56, 52, 44 or 36 (52, 48, 40 or 32 for
// the crossing-map source).
constexpr int kCompactRm = 1, kNarrowRm = 3, kWideRm = 7, kXWideRm = 11;
constexpr int strip_width(bool src_z, int rm_class) { return 58 - 2 * rm_class - (src_z ? 4 : 0); }
constexpr int kDefaultUnitH = 512;
// unit heights the batched plan's autotuner times
constexpr int kNumUnitHeights = 4;
constexpr int kUnitHeights[kNumUnitHeights] = {256, 512, 768, 1024};
constexpr int kMaxCtasPerSm = 32;
// Warps per CTA of the streaming kernels and CTAs per SM of the first pass
// (its __launch_bounds__ and the wave model of the unit height).  One-warp
// CTAs, 13 per SM: a warp's slot frees when its own unit ends, and under the
// bound of 13 x 32 threads the compiler keeps the strip in about 127
// registers without spill.  Measured on a 16384^2 band (specialised kernel):
// 1 x 13 251.8 Gpx/s, 1 x 14 248.3, 1 x 16 249.2, 1 x 12 243.4, 2 x 7 225.0,
// 4 x 3 227.4, 4 x 4 220.4.
#ifndef FX_WARPS_PER_CTA
#define FX_WARPS_PER_CTA 1
#endif
constexpr int kWarpsPerCta = FX_WARPS_PER_CTA;
#ifndef FX_FIRST_PASS_CTAS
#define FX_FIRST_PASS_CTAS 13
#endif
constexpr int kFirstPassCtas = FX_FIRST_PASS_CTAS;
// The batched group kernels carry their queue loop as well: at 13 warps per
// SM (four on some scheduler, so 128 registers) they spill, at 12 (168
// registers) they do not.
#ifndef FX_BATCH_CTAS
#define FX_BATCH_CTAS 12
#endif
constexpr int kBatchCtas = FX_BATCH_CTAS;

// Where the first pass takes the LoG ring weights and the contrast threshold
// from: the kernel parameters (RuntimeConsts), or, in a kernel compiled at run
// time for one parameter set (fx_specialize), compile-time constants that
// become instruction immediates (a packed FP32x2 operand from the parameters
// needs a register pair holding the value twice).
// A kernel compiled for one parameter set also fixes the median list (kNhmf
// levels of windows hmf(l)) and whether loaded values are checked against the
// FP32-exact bound (kCheck).
struct RuntimeConsts {
  static constexpr bool kStatic = false;
  static constexpr int kNhmf = 0;
  static constexpr bool kCheck = false;
  static __device__ __forceinline__ float w(int, int) { return 0.0f; }
  static __device__ __forceinline__ float ntzc(int) { return 0.0f; }
  static __device__ __forceinline__ int hmf(int) { return 0; }
};

inline bool fast_unit_shape_ok(int w, int h, bool src_z) {
  return w == strip_width(src_z, kNarrowRm) && h >= 16 && h <= 8192 && h % 16 == 0;
}
inline size_t fast_smem_bytes(int, int, int) { return 0; }  // static shared memory only

namespace st {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWinCols = 64;
constexpr uint32_t M0 = 0x55555555u, M1 = 0xAAAAAAAAu;  // bits of column 0 / column 1

// Neighbour words: bit of pixel p in the result = bit of its neighbour.
// own = this lane's word, nx / pv = the next / previous lane's word of the same
// rows, nb / pb = this lane's word of the next / previous 16 rows.
__device__ __forceinline__ uint32_t e1(uint32_t o, uint32_t nx) { return ((o >> 1) & M0) | ((nx << 1) & M1); }
__device__ __forceinline__ uint32_t w1(uint32_t o, uint32_t pv) { return ((o << 1) & M1) | ((pv >> 1) & M0); }
__device__ __forceinline__ uint32_t n1(uint32_t o, uint32_t pb) { return __funnelshift_r(o, pb, 2); }
__device__ __forceinline__ uint32_t s1(uint32_t o, uint32_t nb) { return __funnelshift_l(nb, o, 2); }
__device__ __forceinline__ uint32_t n2(uint32_t o, uint32_t pb) { return __funnelshift_r(o, pb, 4); }
__device__ __forceinline__ uint32_t s2(uint32_t o, uint32_t nb) { return __funnelshift_l(nb, o, 4); }
__device__ __forceinline__ uint32_t n3(uint32_t o, uint32_t pb) { return __funnelshift_r(o, pb, 6); }
__device__ __forceinline__ uint32_t s3(uint32_t o, uint32_t nb) { return __funnelshift_l(nb, o, 6); }

__device__ __forceinline__ void fadd(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &k) {
  s = a ^ b ^ c;
  k = (a & b) | (c & (a ^ b));
}
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a | b)); }
// bitwise count of five bits: n = c0 + 2 c1 + 4 c2
__device__ __forceinline__ void count5(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e, uint32_t &c0,
                                       uint32_t &c1, uint32_t &c2) {
  uint32_t s1, k1, k2;
  fadd(a, b, c, s1, k1);
  fadd(d, e, s1, c0, k2);
  c1 = k1 ^ k2;
  c2 = k1 & k2;
}
// bitwise "at least 5 of 9"
__device__ __forceinline__ uint32_t maj9(const uint32_t x[9]) {
  uint32_t s1, c1, s2, c2, s3, c3, s4, c4;
  fadd(x[0], x[1], x[2], s1, c1);
  fadd(x[3], x[4], x[5], s2, c2);
  fadd(x[6], x[7], x[8], s3, c3);
  fadd(s1, s2, s3, s4, c4);
  const uint32_t at2 = (c1 & c2) | (c3 & c4) | ((c1 | c2) & (c3 | c4));
  const uint32_t at3 = (c1 & c2 & (c3 | c4)) | (c3 & c4 & (c1 | c2));
  return at3 | (at2 & s4);
}
// bitwise "at least 7 of 13": weight-1 bits s1..s4 and x[12] counted to
// p0 + 2 p1 + 4 p2, weight-2 carries c1..c4 and p1 to q0 + 2 q1 + 4 q2 (in units
// of 2), so the total is p0 + 2 q0 + 4 (q1 + p2) + 8 q2
__device__ __forceinline__ uint32_t maj13(const uint32_t x[13]) {
  uint32_t s1, c1, s2, c2, s3, c3, s4, c4, p0, p1, p2, q0, q1, q2;
  fadd(x[0], x[1], x[2], s1, c1);
  fadd(x[3], x[4], x[5], s2, c2);
  fadd(x[6], x[7], x[8], s3, c3);
  fadd(x[9], x[10], x[11], s4, c4);
  count5(s1, s2, s3, s4, x[12], p0, p1, p2);
  count5(c1, c2, c3, c4, p1, q0, q1, q2);
  return q2 | (q1 & p2) | ((q1 ^ p2) & q0 & p0);
}
// bitwise "at least 3 of 5"
__device__ __forceinline__ uint32_t maj5(const uint32_t x[5]) {
  uint32_t s1, c1, s2, c2;
  fadd(x[0], x[1], x[2], s1, c1);
  fadd(x[3], x[4], s1, s2, c2);
  return (c1 & c2) | ((c1 | c2) & s2);
}

// Pack the sign bit of v into an accumulator (shift-left insertion).
__device__ __forceinline__ void put(uint32_t &acc, uint32_t v) { acc = __funnelshift_l(v, acc, 1); }

// Arithmetic of a strip.  kModeF32 / kModeInt: integer masks, exact FP32 or
// int32 / int64 arithmetic.  kModeF32Log / kModeF32LogWide: the FP32-LoG mode
// (non-integer masks, L rounded in FP32), with 32-bit or 64-bit sums for the
// exact standard-deviation test.  Values of the lane's two columns travel as
// a pair P: on the FP32 paths a float2, so that every linear operation is one
// packed FP32x2 instruction (IEEE round-to-nearest per element, hence the same
// results as two scalar operations); on the integer path two int32.
enum : int { kModeF32 = 0, kModeInt = 1, kModeF32Log = 2, kModeF32LogWide = 3 };

template <int kMode>
struct Ar;

// FP32 path: values <= fbound, every intermediate an exact FP32 integer.
template <>
struct Ar<kModeF32> {
  static constexpr bool kRel = false;     // L from the ring sums R_c directly
  static constexpr bool kChecked = true;  // values above fbound send the strip to the redo pass
  // Eq. 2 sums of squares are taken over the biased bits K + u (K = 0x4B000000,
  // the bits of the FP32 value u + 2^23) and the bias is removed in sdfail.
  static constexpr bool kBiased = true;
  using V = float;
  using P = float2;
  using Q = uint32_t;
  static __device__ __forceinline__ P mk(V a, V b) { return make_float2(a, b); }
  static __device__ __forceinline__ V lo(P p) { return p.x; }
  static __device__ __forceinline__ V hi(P p) { return p.y; }
  static __device__ __forceinline__ P add(P a, P b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V add1(V a, V b) { return __fadd_rn(a, b); }
  // w x + y (one rounding per element)
  static __device__ __forceinline__ P fma(V w, P x, P y) { return __ffma2_rn(make_float2(w, w), x, y); }
  static __device__ __forceinline__ P zero() { return make_float2(0.0f, 0.0f); }
  static __device__ __forceinline__ V cvt(uint32_t u) { return __uint_as_float(0x4B000000u | u) - 8388608.0f; }
  static __device__ __forceinline__ Q sq(uint32_t u) { return u * u; }
  static __device__ __forceinline__ V w(const KParams &kp, int f, int c) { return kp.ringf[f][c]; }
  static __device__ __forceinline__ uint32_t bits(V x) { return __float_as_uint(x); }
  // 0 - x (+0 for x = 0: no response is ever -0)
  static __device__ __forceinline__ P neg(P x) { return __ffma2_rn(x, make_float2(-1.0f, -1.0f), zero()); }
  static __device__ __forceinline__ V max3(V a, V b, V c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
  }
  static __device__ __forceinline__ V min3(V a, V b, V c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
  }
  // sign bits set  <=>  max - min <= t_zc  (contrast test fails), both columns
  static __device__ __forceinline__ P cfail_c(float ntzc1f, P mx, P mn) {
    const P d = __ffma2_rn(mn, make_float2(-1.0f, -1.0f), mx);  // max - min, rounded once
    return __fadd2_rn(d, make_float2(ntzc1f, ntzc1f));
  }
  static __device__ __forceinline__ P cfail(const KParams &kp, int f, P mx, P mn) {
    return cfail_c(kp.ntzc1f[f], mx, mn);
  }
  // Sign bits set  <=>  the standard-deviation test fails (reading R4), for
  // both columns (A3, A5: pixel sums; Q3, Q5: sums of the squared biased bits).
  // Q = sum (K + u)^2 = sum u^2 + 2K A (mod 2^32, as K^2 = 0), so
  // D = Lambda sum u^2 - A^2 = Lambda Q - b (b + c)  with b = K + A = bits(A + 2^23)
  // and c = 16K (Lambda = 9) or 48K (Lambda = 25); -b - c is the bit pattern of
  // one exact FFMA of A (2^-117 - A 2^-141, resp. A 2^-77 - 2^-53).  D < 2^32.
  // The three threshold tests come out as sign bits (KParams::ntt*) and the
  // gate S = (s5 > t_sdmax) ? (s3 > t_sd3) : (s5 > t_sd5) is a bitwise select.
  static __device__ __forceinline__ void sdfail(const KParams &kp, int f, P A3, P A5, const Q Q3[2],
                                                const Q Q5[2], uint32_t out[2]) {
    const P B3 = __fadd2_rn(A3, make_float2(8388608.0f, 8388608.0f));
    const P B5 = __fadd2_rn(A5, make_float2(8388608.0f, 8388608.0f));
    const P N3 = __ffma2_rn(A3, make_float2(-0x1p-141f, -0x1p-141f), make_float2(0x1p-117f, 0x1p-117f));
    const P N5 = __ffma2_rn(A5, make_float2(0x1p-77f, 0x1p-77f), make_float2(-0x1p-53f, -0x1p-53f));
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t b3 = __float_as_uint(j ? B3.y : B3.x), n3 = __float_as_uint(j ? N3.y : N3.x);
      const uint32_t b5 = __float_as_uint(j ? B5.y : B5.x), n5 = __float_as_uint(j ? N5.y : N5.x);
      const uint32_t r3 = Q3[j] * 9u + (b3 * n3 + kp.ntt3[f]);  // D3 - tt3
      const uint32_t d5 = Q5[j] * 25u + b5 * n5;
      const uint32_t r5 = d5 + kp.ntt5[f], rm = d5 + kp.nttmax[f];  // D5 - tt5, D5 - ttmax
      const uint32_t g = ~d5 & rm;          // bit 31: D5 < ttmax
      out[j] = (g & r5) | (~g & r3);       // bit 31: the selected test fails
    }
  }
};

// Pair of int32 for the integer path.
struct I2 {
  int32_t x, y;
};

// Integer path: any uint16 value (|L| < 2^30 by the plan's range check).
template <>
struct Ar<kModeInt> {
  static constexpr bool kRel = false;
  static constexpr bool kChecked = false;
  static constexpr bool kBiased = false;
  using V = int32_t;
  using P = I2;
  using Q = uint64_t;
  static __device__ __forceinline__ P mk(V a, V b) { return P{a, b}; }
  static __device__ __forceinline__ V lo(P p) { return p.x; }
  static __device__ __forceinline__ V hi(P p) { return p.y; }
  static __device__ __forceinline__ P add(P a, P b) { return P{a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ V add1(V a, V b) { return a + b; }
  static __device__ __forceinline__ P fma(V w, P x, P y) { return P{w * x.x + y.x, w * x.y + y.y}; }
  static __device__ __forceinline__ P zero() { return P{0, 0}; }
  static __device__ __forceinline__ V cvt(uint32_t u) { return static_cast<int32_t>(u); }
  static __device__ __forceinline__ Q sq(uint32_t u) { return static_cast<uint64_t>(u) * u; }
  static __device__ __forceinline__ V w(const KParams &kp, int f, int c) { return kp.ring[f][c]; }
  static __device__ __forceinline__ uint32_t bits(V x) { return static_cast<uint32_t>(x); }
  static __device__ __forceinline__ P neg(P x) { return P{-x.x, -x.y}; }
  static __device__ __forceinline__ V max3(V a, V b, V c) { return max(max(a, b), c); }
  static __device__ __forceinline__ V min3(V a, V b, V c) { return min(min(a, b), c); }
  static __device__ __forceinline__ P cfail(const KParams &kp, int f, P mx, P mn) {
    const uint32_t t = static_cast<uint32_t>(kp.tzc[f]) + 1u;
    return P{static_cast<int32_t>(static_cast<uint32_t>(mx.x - mn.x) - t),
             static_cast<int32_t>(static_cast<uint32_t>(mx.y - mn.y) - t)};
  }
  static __device__ __forceinline__ void sdfail(const KParams &kp, int f, P A3, P A5, const Q Q3[2],
                                                const Q Q5[2], uint32_t out[2]) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int64_t a3 = j ? A3.y : A3.x, a5 = j ? A5.y : A5.x;
      const int64_t d3 = 9 * static_cast<int64_t>(Q3[j]) - a3 * a3;
      const int64_t d5 = 25 * static_cast<int64_t>(Q5[j]) - a5 * a5;
      const bool pass = d5 > kp.tsdmax[f] ? d3 > kp.tsd3[f] : d5 > kp.tsd5[f];
      out[j] = pass ? 0u : 0x80000000u;
    }
  }
};

// FP32-LoG mode, values <= fbound (32-bit standard-deviation sums).  L is
// evaluated from d_c = R_c - n_c I(p) (exact), so flat neighbourhoods give an
// exact 0 and mirrored neighbourhoods exactly opposite responses.
template <>
struct Ar<kModeF32Log> : Ar<kModeF32> {
  static constexpr bool kRel = true;
};

// FP32-LoG mode, any uint16 value: the same FP32 responses, 64-bit D.
template <>
struct Ar<kModeF32LogWide> : Ar<kModeF32> {
  static constexpr bool kRel = true;
  static constexpr bool kChecked = false;
  static constexpr bool kBiased = false;
  using Q = uint64_t;
  static __device__ __forceinline__ Q sq(uint32_t u) { return static_cast<uint64_t>(u) * u; }
  static __device__ __forceinline__ void sdfail(const KParams &kp, int f, P A3, P A5, const Q Q3[2],
                                                const Q Q5[2], uint32_t out[2]) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      // A3, A5 are exact integers below 2^21
      const int64_t a3 = static_cast<int64_t>(__float_as_uint((j ? A3.y : A3.x) + 8388608.0f) - 0x4B000000u);
      const int64_t a5 = static_cast<int64_t>(__float_as_uint((j ? A5.y : A5.x) + 8388608.0f) - 0x4B000000u);
      const int64_t d3 = 9 * static_cast<int64_t>(Q3[j]) - a3 * a3;
      const int64_t d5 = 25 * static_cast<int64_t>(Q5[j]) - a5 * a5;
      const bool pass = d5 > kp.tsdmax[f] ? d3 > kp.tsd3[f] : d5 > kp.tsd5[f];
      out[j] = pass ? 0u : 0x80000000u;
    }
  }
};

// kPair: one aligned load of the lane's two pixels per row (images whose base
// and pitch are multiples of two pixels and whose width is even); otherwise
// two single-pixel loads.  Either way every load is unconditional and lands in
// a ring slot that is read four steps later, so loads overlap the arithmetic;
// the clamped (replicated, reading R2) columns are selected when a row is used.
// kSd2: the branches have different standard-deviation thresholds (two S words).
// kSrcZ: the standard deviation is taken over each branch's crossing map
// (reading R4, source 1) from bit-sliced counts, at block level.
// kRm: the strip class (kCompactRm, kNarrowRm, kWideRm or kXWideRm): the
// halo, and for the wide classes the ring prefill one (two) iterations
// earlier, so that the rows above the unit that the outputs depend on are
// computed (the mask rows down to r above the unit).
// Cst: RuntimeConsts, or the constants of a run-time compiled kernel (FP32
// modes only).
template <typename T, int kMode, bool kPair, bool kSd2, bool kSrcZ, int kRm = kNarrowRm, class Cst = RuntimeConsts>
struct Strip {
  using A = Ar<kMode>;
  // halo columns left of the strip (even: the pair loads are aligned) and
  // output columns: 2 LoG + 1 crossing (+ 2 standard deviation) + kRm median
  static constexpr int kLeftHalo = 3 + kRm + (kSrcZ ? 2 : 0), kOutCols = strip_width(kSrcZ, kRm);
  static_assert(2 * kLeftHalo + kOutCols == 64 && kLeftHalo % 2 == 0, "symmetric, even halo");
  // first iteration (rows 4 kK0 .. are the ring prefill): the mask is valid
  // from 3 rows below the first prefill row, so down to 4 |kK0| - 3 rows above
  // the unit (block -1, from 19 rows above, holds them)
  static constexpr int kK0 = kRm > kWideRm ? -4 : kRm > kNarrowRm ? -3 : -2;
  static_assert(4 * -kK0 - 3 >= kRm, "the prefill reaches the rows the medians need");
  using V = typename A::V;
  using P = typename A::P;
  using Q = typename A::Q;

  const ImageView &v;
  const KParams &kp;
  int64_t X0, Y0, Y1, xs, W, H;
  int lane;
  bool check, border, vstore;
  int bl_lane, bl_slot, br_lane, br_slot;
  uint32_t outmask_l, outmask_r;  // this lane's slots left of / right of the image (M0 << j)

  // Rings of period 4 (slot of row t = t & 3), one pair (the lane's two
  // columns) per row.  The row four steps back is read before the newest row
  // overwrites its slot; sums over it are taken first, so that the new row can
  // take its registers.
  P f_[4], h1_[4], h2_[4];
  Q c3_[4][2], c5_[4][2];
  P L_[2][4];
  uint32_t S_[2][4][2];  // sign bit: the standard-deviation test fails
  uint32_t raw_[4], raw1_[4];  // loaded pixels of rows t..t+3 (raw1_: second pixel, !kPair)
  uint32_t vmax_;
  uint32_t vhi_;  // 0 when the high half of this lane's loaded pair is padding (odd width)
  uint32_t acc_[12];
  // Words of earlier blocks, touched once per 16 rows, live in shared memory:
  // kBlk.. = previous block (12 words), kPneg / kPpos / kPsS = neg / pos / sS of
  // the block before it, kLev + 2l / + 2l + 1 = the words of median level l
  // (level 0: the mask M) of the two blocks before, kZA / kZB = crossing words
  // of the two blocks before and kPcf = contrast words of the block before
  // (kSrcZ).
  uint32_t (*sw_)[32];
  static constexpr int kBlk = 0, kPneg = 12, kPpos = 14, kPsS = 16, kLev = 18, kMA = kLev, kZA = 26, kZB = 28,
                       kPcf = 30, kWords = 32;
  // kAsync (the FP32 paths): the input rows arrive in an 8-row ring of words
  // in shared memory (kRing .. kRing + 7), filled by cp.async seven rows
  // ahead, so loads in flight hold no registers.  With kPair a lane's word is
  // its uint16 pair, or for uint8 the aligned 4-byte word holding its pair.
  // Without (kTwoWord: base or pitch not a multiple of 4 bytes) a lane copies
  // the aligned 4-byte word holding its first pixel and, when its pixels run
  // past that word, the next one into a second ring (kRing2 .. kRing2 + 7);
  // the row's byte offset selects the pixels (each word holds an image byte,
  // so it lies in that byte's page).
  static constexpr bool kAsync = A::kBiased;
  static constexpr bool kTwoWord = kAsync && !kPair;
  static constexpr int kRing = kWords, kRingRows = 8, kRing2 = kWords + kRingRows;
  static constexpr uint32_t kRing2Off = 128u * kRingRows;  // bytes from a ring word to its second-ring word
  __device__ __forceinline__ uint32_t &blk(int i) { return sw_[kBlk + i][lane]; }

  // load state: rows relative to Y0; p0_ / p1_ address row rbase
  int32_t rlo, rhi, Hrel, Y0rel, rbase;
  const unsigned char *p0_, *p1_;
  uint32_t pitch32;
  uint32_t sel_;  // kPair: byte selector taking the clamped columns out of the loaded pair
  // byte selectors making the biased bits K + u of the lane's two pixels from
  // the loaded word(s) and K (A::kBiased)
  uint32_t selb0_, selb1_;
  // kAsync: shared-memory address of this lane's word in ring slot 4 (k & 1)
  // (slots 4 (k & 1) + S hold the rows of iteration k) and in the other half
  uint32_t ring_h_, ring_o_;
  // FX_CHECKED: the ring's first slot, and whether this lane's loaded
  // column(s) lie in the row (the image, or the padding element after column
  // W - 1 of an odd-width row with pitch slack)
  uint32_t ring_base_;
  bool colok_;
  // kTwoWord: pixel-selector base (byte offset 0) and bytes the lane's pixels span
  uint32_t psel_c_, span_;

  __device__ Strip(const ImageView &v_, const KParams &kp_, int64_t x0, int64_t y0, int64_t y1,
                   uint32_t (*words)[32])
      : v(v_), kp(kp_), X0(x0), Y0(y0), Y1(y1), sw_(words) {
    lane = threadIdx.x & 31;
    W = v.width;
    H = v.height;
    xs = X0 - kLeftHalo;
    check = Cst::kStatic ? Cst::kCheck : A::kChecked && kp.fbound < (sizeof(T) == 1 ? 255 : 65535);
    border = xs < 0 || xs + kWinCols > W;
    vstore = (reinterpret_cast<uintptr_t>(v.out) % 2 == 0) && (v.out_pitch % 2 == 0) && (xs % 2 == 0);
    const int64_t bl = -xs, br = W - 1 - xs;  // window columns of image columns 0 and W-1
    bl_lane = bl > 0 ? static_cast<int>(bl >> 1) : 0;
    bl_slot = bl > 0 ? static_cast<int>(bl & 1) : 0;
    br_lane = br < kWinCols - 1 ? static_cast<int>((br < 0 ? 0 : br) >> 1) : 31;
    br_slot = br < kWinCols - 1 ? static_cast<int>((br < 0 ? 0 : br) & 1) : 1;
    outmask_l = outmask_r = 0;
    const int64_t x = xs + 2 * lane;
    for (int j = 0; j < 2; ++j) {
      if (x + j < 0) outmask_l |= M0 << j;
      if (x + j >= W) outmask_r |= M0 << j;
    }
    const int64_t lo = v.row0 > 0 ? v.row0 : 0, hi = (v.row_lim < H ? v.row_lim : H) - 1;
    rlo = static_cast<int32_t>(lo - Y0);
    rhi = static_cast<int32_t>(hi - Y0);
    Hrel = static_cast<int32_t>(H - Y0);
    Y0rel = static_cast<int32_t>(Y0 < (1 << 30) ? Y0 : (1 << 30));
    // rows a unit reads are >= Y0 + 4 kK0 (the first prefill row) and >= the
    // buffer's first row; load offsets count from there, so they are never
    // negative
    rbase = rlo > 4 * kK0 ? rlo : 4 * kK0;
    pitch32 = static_cast<uint32_t>(v.pitch);
    const unsigned char *base = static_cast<const unsigned char *>(v.img) + (Y0 + rbase - v.row0) * v.pitch;
    const int64_t d0 = x < 0 ? 0 : (x >= W ? W - 1 : x), d1 = x + 1 < 0 ? 0 : (x + 1 >= W ? W - 1 : x + 1);
    vhi_ = 0xFFFFu;
    if constexpr (kPair) {
      // the even pair (cb, cb + 1) inside the row that holds both clamped
      // columns; for an odd width the last column's pair is (W - 1, W), W being
      // the first padding element of the row
      const int64_t we = W + (W & 1);
      const int64_t cb = (d0 < we - 2 ? d0 : we - 2) & ~int64_t{1};
      if (cb + 1 >= W) vhi_ = 0;
      // the loaded word: the pair itself (uint16), or the aligned 4-byte word
      // holding it (uint8; the row pitch reaches the end of that word)
      const int64_t ca = sizeof(T) == 1 ? (cb & ~int64_t{3}) : cb;
      colok_ = cb >= 0 && (cb + 1 < W || (cb + 1 == W && v.pitch >= (W + 1) * static_cast<int64_t>(sizeof(T)))) &&
               (sizeof(T) == 2 || ca + 4 <= v.pitch);
      p0_ = p1_ = base + ca * static_cast<int64_t>(sizeof(T));
      const uint32_t h0 = static_cast<uint32_t>(d0 - ca), h1 = static_cast<uint32_t>(d1 - ca);
      if constexpr (sizeof(T) == 2) {
        sel_ = (h0 ? 0x32u : 0x10u) | ((h1 ? 0x32u : 0x10u) << 8);
        selb0_ = h0 ? 0x7432u : 0x7410u;
        selb1_ = h1 ? 0x7432u : 0x7410u;
      } else {
        sel_ = h0 | 0x40u | (h1 << 8) | 0x4000u;
        selb0_ = 0x7440u | h0;
        selb1_ = 0x7440u | h1;
      }
    } else {
      p0_ = base + d0 * static_cast<int64_t>(sizeof(T));
      p1_ = base + d1 * static_cast<int64_t>(sizeof(T));
      colok_ = d0 >= 0 && d0 < W && d1 >= 0 && d1 < W;
      sel_ = 0x5410u;
      selb0_ = selb1_ = 0x7410u;  // each load holds one zero-extended pixel
      if constexpr (kTwoWord) {
        // the pixels as a pair word: bytes (o, o + 1, o + 2 dl, o + 2 dl + 1) of
        // the two words for uint16, (o, o + dl, o, o) for uint8, o being the
        // row's byte offset in the first word and dl = d1 - d0 (0 at a border)
        const uint32_t dl = static_cast<uint32_t>(d1 - d0);
        psel_c_ = sizeof(T) == 2 ? (0x0010u | ((2u * dl) << 8) | ((2u * dl + 1u) << 12)) : (dl << 4);
        span_ = static_cast<uint32_t>(sizeof(T)) * (1u + dl);
        selb0_ = sizeof(T) == 2 ? 0x7410u : 0x7440u;
        selb1_ = sizeof(T) == 2 ? 0x7432u : 0x7441u;
      } else {
        psel_c_ = span_ = 0;
      }
    }
    vmax_ = 0;
    for (int i = 0; i < 12; ++i) acc_[i] = 0;
    for (int i = 0; i < kWords; ++i) sw_[i][lane] = 0;
    ring_h_ = ring_o_ = ring_base_ = static_cast<uint32_t>(__cvta_generic_to_shared(&sw_[kRing][lane]));
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      f_[s] = h1_[s] = h2_[s] = A::zero();
      L_[0][s] = L_[1][s] = A::zero();
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        c3_[s][j] = c5_[s][j] = Q(0);
        S_[0][s][j] = S_[1][s][j] = 0;
      }
      raw_[s] = raw1_[s] = 0;
    }
  }

  // LoG ring weight c of mask f, and the contrast test (sign bits set <=>
  // max - min <= t_zc) of branch f
  __device__ __forceinline__ V wgt(int f, int c) const {
    if constexpr (Cst::kStatic) return static_cast<V>(Cst::w(f, c));
    else return A::w(kp, f, c);
  }
  __device__ __forceinline__ P cfail(int f, P mx, P mn) const {
    if constexpr (Cst::kStatic) return A::cfail_c(Cst::ntzc(f), mx, mn);
    else return A::cfail(kp, f, mx, mn);
  }
  // the median list and the bound check, fixed or from the parameters
  __device__ __forceinline__ int nhmf() const { return Cst::kStatic ? Cst::kNhmf : kp.nhmf; }
  __device__ __forceinline__ int hmf_at(int l) const { return Cst::kStatic ? Cst::hmf(l) : kp.hmf[l]; }
  __device__ __forceinline__ bool checking() const { return Cst::kStatic ? Cst::kCheck : check; }

  // Row t (relative to Y0) into ring slot S.  Rows outside the image clamp to
  // it (reading R2); rows outside the buffer (a row band) clamp to the buffer:
  // they feed only rows that are not stored.
  template <int S, bool kClamp = true>
  __device__ __forceinline__ void load_row(int32_t tr) {
    const int32_t yr = kClamp ? (tr < rlo ? rlo : (tr > rhi ? rhi : tr)) : tr;
    const uint64_t off = static_cast<uint64_t>(static_cast<uint32_t>(yr - rbase)) * pitch32;
    if (!FX_GUARD(yr >= rlo && yr <= rhi && yr >= rbase && colok_)) return;
    if constexpr (kPair) {
      raw_[S] = __ldg(reinterpret_cast<const uint32_t *>(p0_ + off));  // the lane's word (see kAsync)
    } else {
      raw_[S] = __ldg(reinterpret_cast<const T *>(p0_ + off));
      raw1_[S] = __ldg(reinterpret_cast<const T *>(p1_ + off));
    }
  }

  // kAsync: row t (relative to Y0) into the ring word at shared address dst
  // (clamped like load_row), as one cp.async commit group.
  template <bool kClamp = true>
  __device__ __forceinline__ void load_row_async(uint32_t dst, int32_t tr) {
    const int32_t yr = kClamp ? (tr < rlo ? rlo : (tr > rhi ? rhi : tr)) : tr;
    const uint64_t off = static_cast<uint64_t>(static_cast<uint32_t>(yr - rbase)) * pitch32;
    if (!FX_GUARD(yr >= rlo && yr <= rhi && yr >= rbase && colok_ && dst - ring_base_ < 128u * kRingRows &&
                  (dst - ring_base_) % 128u == 0)) {
      asm volatile("cp.async.commit_group;" ::: "memory");  // an empty group keeps the wait counts
      return;
    }
    if constexpr (kTwoWord) {
      const unsigned char *a = p0_ + off;
      const uint32_t o = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(a)) & 3u;
      const unsigned char *w = a - o;  // the aligned word holding the first pixel
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(w) : "memory");
      if (o + span_ > 4u)  // the pixels run into the next word
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + kRing2Off), "l"(w + 4) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n\tcp.async.commit_group;" ::"r"(dst), "l"(p0_ + off)
                   : "memory");
    }
  }
  __device__ __forceinline__ void async_drain() {
    if constexpr (kAsync) asm volatile("cp.async.wait_group 0;" ::: "memory");
  }

  // Running maximum of the loaded values (the FP32 bound check): per 16-bit
  // half for uint16 words, per byte for uint8 (a word may hold the
  // neighbouring lane's pair too, which only makes the check conservative).
  __device__ __forceinline__ void track_max(uint32_t w) {
    vmax_ = sizeof(T) == 1 ? __vmaxu4(vmax_, w) : __vmaxu2(vmax_, w);
  }
  __device__ __forceinline__ uint32_t tracked_max() const {
    if constexpr (sizeof(T) == 1)
      return max(max(vmax_ & 0xFFu, (vmax_ >> 8) & 0xFFu), max((vmax_ >> 16) & 0xFFu, vmax_ >> 24));
    else
      return max(vmax_ & 0xFFFFu, (vmax_ >> 16) & vhi_);
  }

  // The lane's two pixels of the row in slot S as a 16-bit pair (column 0 low).
  // (The selection also copies the ring slot before the next load refills it;
  // reading the slot directly made that load wait on its predecessor's use.)
  template <int S>
  __device__ __forceinline__ uint32_t pixels() const {
    if constexpr (kPair) return __byte_perm(raw_[S], 0, sel_);
    else return __byte_perm(raw_[S], raw1_[S], 0x5410);
  }

  // Replace the values of window columns outside the image by the value of the
  // nearest image column (reading R2 for a stage array).
  __device__ __forceinline__ void fix_cols(V x[2]) {
    const V sl = bl_slot == 0 ? x[0] : x[1];
    const V sr = br_slot == 0 ? x[0] : x[1];
    const V lv = __shfl_sync(kFull, sl, bl_lane);
    const V rv = __shfl_sync(kFull, sr, br_lane);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (outmask_l & (M0 << j)) x[j] = lv;
      if (outmask_r & (M0 << j)) x[j] = rv;
    }
  }

  __device__ __forceinline__ void fix_cols(P &x) {
    V a[2] = {A::lo(x), A::hi(x)};
    fix_cols(a);
    x = A::mk(a[0], a[1]);
  }

  // Same for a mask word: columns outside the image take the border column's bits.
  __device__ __forceinline__ uint32_t fix_cols_bits(uint32_t m) {
    const uint32_t ml = __shfl_sync(kFull, m, bl_lane);
    const uint32_t mr = __shfl_sync(kFull, m, br_lane);
    const uint32_t repl = ((ml >> bl_slot) & M0) * 0x3u;
    const uint32_t repr = ((mr >> br_slot) & M0) * 0x3u;
    m = (m & ~outmask_l) | (repl & outmask_l);
    m = (m & ~outmask_r) | (repr & outmask_r);
    return m;
  }

  // kChk: the step may need the border fix-ups of the L stage (a border strip,
  // or rows next to the first or last image row); otherwise they are no-ops.
  template <int S, bool kChk>
  __device__ __forceinline__ void step(int32_t t) {  // t relative to Y0, S = t & 3
    constexpr int c0 = (S + 2) & 3, m1 = (S + 1) & 3, p1 = (S + 3) & 3;  // rows t-2, t-3, t-1
    // Row t: F = the lane's two pixels (columns 0, 1), Fl / Fr = columns -2, -1
    // / 2, 3 (the neighbouring lanes' pixels), c3n / c5n = the 3- and 5-wide
    // sums of squares per column.
    P F, Fl, Fr;
    Q c3n[2] = {}, c5n[2] = {};
    if constexpr (A::kBiased) {
      // biased bits K + u (K = 0x4B000000; FP32 value u + 2^23) straight from the
      // loaded word(s), before the load ahead refills the slot
      uint32_t r0, r1;
      if constexpr (kAsync) {
        // row t is in ring slot t & 7 = 4 (k & 1) + S; six younger rows may be in flight
        r0 = 0;
        if (FX_GUARD(ring_h_ + 128u * S - ring_base_ < 128u * kRingRows))
          asm volatile("cp.async.wait_group 6;\n\tld.shared.u32 %0, [%1];" : "=r"(r0) : "r"(ring_h_ + 128u * S) : "memory");
        r1 = r0;
        if constexpr (kTwoWord) {
          // the row's byte offset (its load clamped the row the same way)
          uint32_t w1 = 0;
          if (FX_GUARD(ring_h_ + 128u * S - ring_base_ < 128u * kRingRows))
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w1) : "r"(ring_h_ + 128u * S + kRing2Off) : "memory");
          const int32_t yr = t < rlo ? rlo : (t > rhi ? rhi : t);
          const uint32_t o = (static_cast<uint32_t>(reinterpret_cast<uintptr_t>(p0_)) +
                              static_cast<uint32_t>(yr - rbase) * pitch32) & 3u;
          r0 = __byte_perm(r0, w1, psel_c_ + o * 0x1111u);  // the pixels as a pair word
          r1 = r0;
        }
        // refill the slot of row t - 1 (read one step ago) with row t + 7
        load_row_async<kChk>(S == 0 ? ring_o_ + 384u : ring_h_ + 128u * (S - 1), t + kRingRows - 1);
      } else {
        r0 = raw_[S];
        r1 = raw1_[S];
      }
      const uint32_t b2 = __byte_perm(r0, 0x4B000000u, selb0_);
      const uint32_t b3 = __byte_perm(kPair || kTwoWord ? r0 : r1, 0x4B000000u, selb1_);
      if (checking()) track_max(kPair || kTwoWord ? r0 : __byte_perm(r0, r1, 0x5410));
      if constexpr (!kAsync) load_row<S, kChk>(t + 4);
      const uint32_t b0 = __shfl_up_sync(kFull, b2, 1), b1 = __shfl_up_sync(kFull, b3, 1);
      const uint32_t b4 = __shfl_down_sync(kFull, b2, 1), b5 = __shfl_down_sync(kFull, b3, 1);
      const P bias = A::mk(-8388608.0f, -8388608.0f);
      F = A::add(A::mk(__uint_as_float(b2), __uint_as_float(b3)), bias);
      Fl = A::add(A::mk(__uint_as_float(b0), __uint_as_float(b1)), bias);
      Fr = A::add(A::mk(__uint_as_float(b4), __uint_as_float(b5)), bias);
      if constexpr (!kSrcZ) {
        const uint32_t s23 = b2 * b2 + b3 * b3;
        c3n[0] = b1 * b1 + s23;
        c3n[1] = b4 * b4 + s23;
        c5n[0] = b0 * b0 + (b4 * b4 + c3n[0]);
        c5n[1] = b5 * b5 + (b1 * b1 + c3n[1]);
      }
    } else {
      const uint32_t w = pixels<S>();
      load_row<S, kChk>(t + 4);  // four rows ahead, into the slot just read
      if (checking()) track_max(w);
      const uint32_t hl = __shfl_up_sync(kFull, w, 1);    // columns -2, -1
      const uint32_t hr = __shfl_down_sync(kFull, w, 1);  // columns 2, 3
      const uint32_t u[6] = {hl & 0xFFFFu, hl >> 16, w & 0xFFFFu, w >> 16, hr & 0xFFFFu, hr >> 16};
      Fl = A::mk(A::cvt(u[0]), A::cvt(u[1]));
      F = A::mk(A::cvt(u[2]), A::cvt(u[3]));
      Fr = A::mk(A::cvt(u[4]), A::cvt(u[5]));
      if constexpr (!kSrcZ) {
        Q sq[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) sq[k] = A::sq(u[k]);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          c3n[j] = sq[j + 1] + sq[j + 2] + sq[j + 3];
          c5n[j] = c3n[j] + sq[j] + sq[j + 4];
        }
      }
    }
    // Sums over row t - 4 (slot S), taken before row t takes its slot.
    const P T4 = A::add(h2_[c0], f_[S]);                     // R4 without row t
    const P T5 = A::add(A::add(h2_[m1], h2_[p1]), h1_[S]);   // R5 without row t
    const P T8 = A::add(h2_[S], Fl);                         // R8 without column +2 of row t
    Q P5[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) P5[j] = c5_[S][j] + c5_[m1][j] + c5_[c0][j];
    // horizontal sums of row t: h1 = I(x-1) + I(x+1), h2 = I(x-2) + I(x+2)
    f_[S] = F;
    h1_[S] = A::mk(A::add1(A::hi(Fl), A::hi(F)), A::add1(A::lo(F), A::lo(Fr)));
    h2_[S] = A::add(Fl, Fr);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      c3_[S][j] = c3n[j];
      c5_[S][j] = c5n[j];
    }
    centre<S, kChk>(t - 2, T4, T5, A::add(T8, Fr), P5);
    pack<S>();
  }

  // LoG responses and the standard-deviation test for the centre row c = t - 2
  // (row t is in slot S; T4 / T5 / R8: the sums that involve row t - 4).
  template <int S, bool kChk>
  __device__ __forceinline__ void centre(int32_t c, P T4, P T5, P R8, const Q P5[2]) {
    constexpr int c0 = (S + 2) & 3, m1 = (S + 1) & 3, p1 = (S + 3) & 3;
    // the six ring sums (squared radii 0, 1, 2, 4, 5, 8) of the radial masks
    const P R0 = f_[c0];
    const P R1 = A::add(h1_[c0], A::add(f_[m1], f_[p1]));
    const P R2 = A::add(h1_[m1], h1_[p1]);
    const P R4 = A::add(T4, f_[S]);
    const P R5 = A::add(T5, h1_[S]);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      if constexpr (A::kRel) {
        // FP32-LoG: one rounding per product-add, in the order of the ring radii
        const P d1 = A::fma(-4.0f, R0, R1), d2 = A::fma(-4.0f, R0, R2);
        const P d4 = A::fma(-4.0f, R0, R4), d5 = A::fma(-8.0f, R0, R5);
        const P d8 = A::fma(-4.0f, R0, R8);
        // starting from +0: a zero product gives +0, so no sum is ever -0
        P l = A::fma(wgt(f, 1), d1, A::zero());
        l = A::fma(wgt(f, 2), d2, l);
        l = A::fma(wgt(f, 3), d4, l);
        l = A::fma(wgt(f, 4), d5, l);
        L_[f][c0] = A::fma(wgt(f, 5), d8, l);
      } else {
        // exact partial sums; starting from +0 no sum is ever -0 (the sign bit
        // of L is the sign of the response)
        P l = A::fma(wgt(f, 0), R0, A::zero());
        l = A::fma(wgt(f, 1), R1, l);
        l = A::fma(wgt(f, 2), R2, l);
        l = A::fma(wgt(f, 3), R4, l);
        l = A::fma(wgt(f, 4), R5, l);
        L_[f][c0] = A::fma(wgt(f, 5), R8, l);
      }
    }
    if constexpr (!kSrcZ) {
      const P A3 = A::add(A::add(R0, R1), R2);
      const P A5 = A::add(A::add(A::add(A3, R4), R5), R8);
      Q Q3[2], Q5[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        Q3[j] = c3_[m1][j] + c3_[c0][j] + c3_[p1][j];
        Q5[j] = P5[j] + c5_[p1][j] + c5_[S][j];
      }
      A::sdfail(kp, 0, A3, A5, Q3, Q5, S_[0][c0]);
      if (kSd2) A::sdfail(kp, 1, A3, A5, Q3, Q5, S_[1][c0]);
    }
    // replicated borders for the L stage (reading R2)
    if constexpr (kChk) {
      if (c >= Hrel) {
#pragma unroll
        for (int f = 0; f < 2; ++f) L_[f][c0] = L_[f][m1];
      }
      if (border) {
        fix_cols(L_[0][c0]);
        fix_cols(L_[1][c0]);
      }
      if (c == -Y0rel) {
#pragma unroll
        for (int f = 0; f < 2; ++f) L_[f][m1] = L_[f][c0];
      }
    }
  }

  // Bits of row c' = t - 3 (its south neighbour row t - 2 is now known).
  template <int S>
  __device__ __forceinline__ void pack() {
    constexpr int r = (S + 1) & 3, rn = S, rs = (S + 2) & 3;  // rows t-3, t-4, t-2
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const P Lc = L_[f][r], Ln = L_[f][rn], Ls = L_[f][rs];
      // west / east neighbours of the lane's columns 0 / 1: the neighbouring lanes'
      const V Lw = __shfl_up_sync(kFull, A::hi(Lc), 1), Le = __shfl_down_sync(kFull, A::lo(Lc), 1);
      const V c0v = A::lo(Lc), c1v = A::hi(Lc);
      const P nL = A::neg(Lc);
      const P sS = A::add(Lc, Ls);
      const V sE0 = A::add1(c0v, c1v), sE1 = A::add1(c1v, Le);
      const P mx = A::mk(A::max3(A::max3(Lw, c0v, c1v), A::lo(Ln), A::lo(Ls)),
                         A::max3(A::max3(c0v, c1v, Le), A::hi(Ln), A::hi(Ls)));
      const P mn = A::mk(A::min3(A::min3(Lw, c0v, c1v), A::lo(Ln), A::lo(Ls)),
                         A::min3(A::min3(c0v, c1v, Le), A::hi(Ln), A::hi(Ls)));
      const P cf = cfail(f, mx, mn);
      // column 1 first: bit 30 - 2r + j for row r, column j
      put(acc_[5 * f + 0], A::bits(c1v));
      put(acc_[5 * f + 0], A::bits(c0v));
      put(acc_[5 * f + 1], A::bits(A::hi(nL)));
      put(acc_[5 * f + 1], A::bits(A::lo(nL)));
      put(acc_[5 * f + 2], A::bits(sE1));
      put(acc_[5 * f + 2], A::bits(sE0));
      put(acc_[5 * f + 3], A::bits(A::hi(sS)));
      put(acc_[5 * f + 3], A::bits(A::lo(sS)));
      put(acc_[5 * f + 4], A::bits(A::hi(cf)));
      put(acc_[5 * f + 4], A::bits(A::lo(cf)));
    }
    if constexpr (kSrcZ) return;
    put(acc_[10], S_[0][r][1]);
    put(acc_[10], S_[0][r][0]);
    if (kSd2) {
      put(acc_[11], S_[1][r][1]);
      put(acc_[11], S_[1][r][0]);
    }
  }

  // Zero crossings (Sec. 3.2, reading R3) of branch f in block g - 1 (words blk;
  // the row below from acc_, the row above from the kP* words).
  __device__ __forceinline__ uint32_t crossings(int f) {
    const uint32_t neg = blk(5 * f), pos = blk(5 * f + 1), sE = blk(5 * f + 2), sS = blk(5 * f + 3);
    const uint32_t negP = __shfl_up_sync(kFull, neg, 1), negX = __shfl_down_sync(kFull, neg, 1);
    const uint32_t posP = __shfl_up_sync(kFull, pos, 1), posX = __shfl_down_sync(kFull, pos, 1);
    const uint32_t sEP = __shfl_up_sync(kFull, sE, 1);
    const uint32_t nE = e1(neg, negX), pE = e1(pos, posX), nW = w1(neg, negP), pW = w1(pos, posP);
    const uint32_t nN = n1(neg, sw_[kPneg + f][lane]), pN = n1(pos, sw_[kPpos + f][lane]);
    const uint32_t nS = s1(neg, acc_[5 * f]), pS = s1(pos, acc_[5 * f + 1]);
    const uint32_t sW = w1(sE, sEP), sN = n1(sS, sw_[kPsS + f][lane]);
    // crossing with each neighbour, and losing it: the pixel wins an edge iff
    // it is the negative one XOR the edge sum is negative (reading R3)
    const uint32_t xE = (neg & pE) | (pos & nE), xW = (neg & pW) | (pos & nW);
    const uint32_t xN = (neg & pN) | (pos & nN), xS = (neg & pS) | (pos & nS);
    const uint32_t lE = xE & ~(neg ^ sE), lW = xW & ~(neg ^ sW);
    const uint32_t lN = xN & ~(neg ^ sN), lS = xS & ~(neg ^ sS);
    const uint32_t znz = (xE | xW | xN | xS) & ~(lE | lW | lN | lS);
    const uint32_t z0 = ~(neg | pos) & ((nW & pE) | (pW & nE) | (nN & pS) | (pN & nS));
    return znz | z0;
  }

  // Block b = g - 1 (image-source standard deviation): extraction and OR (the mask M).
  __device__ __forceinline__ uint32_t mask_block(int64_t b) {
    uint32_t m = 0;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const uint32_t sdf = kSd2 ? blk(10 + f) : blk(10);  // standard-deviation test fails
      m |= crossings(f) & ~(blk(5 * f + 4) | sdf);
    }
    return replicate(b, m, sw_[kMA][lane]);
  }

  // Bit-sliced n >= lo and n <= hi for the NB-bit counts n (planes n[0] = LSB);
  // sel[i] / sel[NB + i] = all ones where bit i of lo / hi is set.
  template <int NB>
  __device__ __forceinline__ static uint32_t in_range(const uint32_t (&n)[NB], const uint32_t *sel) {
    uint32_t ge = 0xFFFFFFFFu, le = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      ge = (sel[i] & n[i] & ge) | (~sel[i] & (n[i] | ge));
      le = (sel[NB + i] & (~n[i] | le)) | (~sel[NB + i] & ~n[i] & le);
    }
    return ge & le;
  }

  // Eq. 2 over the binary crossing map of branch f (reading R4, source 1) for
  // block own (prev / next: the blocks above / below).  With n crossings in a
  // window of Lambda pixels, D = n (Lambda - n); each test D > t holds on an
  // interval of n, precomputed on the host (KParams::zsel).
  __device__ __forceinline__ uint32_t sd_over_z(uint32_t prev, uint32_t own, uint32_t next, int f) {
    // vertical 3- and 5-row sums: t = (t1 t0), v = (v2 v1 v0)
    const uint32_t a = n1(own, prev), c = s1(own, next), d = n2(own, prev), e = s2(own, next);
    uint32_t t0, t1, v0, k1;
    fadd(a, own, c, t0, t1);
    fadd(t0, d, e, v0, k1);
    const uint32_t v1 = t1 ^ k1, v2 = t1 & k1;
    // the same sums of the neighbour lanes (two columns over) and one column over
    const uint32_t t0P = __shfl_up_sync(kFull, t0, 1), t0X = __shfl_down_sync(kFull, t0, 1);
    const uint32_t t1P = __shfl_up_sync(kFull, t1, 1), t1X = __shfl_down_sync(kFull, t1, 1);
    const uint32_t v0P = __shfl_up_sync(kFull, v0, 1), v0X = __shfl_down_sync(kFull, v0, 1);
    const uint32_t v1P = __shfl_up_sync(kFull, v1, 1), v1X = __shfl_down_sync(kFull, v1, 1);
    const uint32_t v2P = __shfl_up_sync(kFull, v2, 1), v2X = __shfl_down_sync(kFull, v2, 1);
    // 3x3 count: t(x-1) + t(x) + t(x+1), 4 bits
    uint32_t x0, x1, y0, y1;
    fadd(w1(t0, t0P), t0, e1(t0, t0X), x0, x1);
    fadd(w1(t1, t1P), t1, e1(t1, t1X), y0, y1);
    const uint32_t cc = x1 & y0;
    const uint32_t n3[4] = {x0, x1 ^ y0, y1 ^ cc, y1 & cc};
    // 5x5 count: v(x-2) + ... + v(x+2), 5 bits; each plane's five bits counted first
    uint32_t p0, p1, p2, q0, q1, q2, r0, r1, r2;
    count5(v0P, w1(v0, v0P), v0, e1(v0, v0X), v0X, p0, p1, p2);
    count5(v1P, w1(v1, v1P), v1, e1(v1, v1X), v1X, q0, q1, q2);
    count5(v2P, w1(v2, v2P), v2, e1(v2, v2X), v2X, r0, r1, r2);
    // total = p0 + 2 (p1 + q0) + 4 (p2 + q1 + r0) + 8 (q2 + r1) + 16 r2
    const uint32_t h1 = p1 ^ q0, hc = p1 & q0;
    uint32_t s4, k4, g4, m4;
    fadd(p2, q1, r0, s4, k4);     // weight 4 (carry k4 to 8)
    const uint32_t t4 = s4 ^ hc;  // with the weight-2 carry
    g4 = s4 & hc;                 // carry to 8
    uint32_t s8, k8;
    fadd(q2, r1, k4, s8, k8);     // weight 8 (carry k8 to 16)
    const uint32_t u8 = s8 ^ g4;
    m4 = s8 & g4;                 // carry to 16
    const uint32_t n5[5] = {p0, h1, t4, u8, r2 ^ k8 ^ m4};  // the count is at most 25
    const uint32_t *sel = kp.zsel[f];
    const uint32_t p5 = in_range(n5, sel), pm = in_range(n5, sel + 10);
    const uint32_t p3 = in_range(n3, sel + 20);
    return (pm & p3) | (~pm & p5);
  }

  // Replicated borders of a binary stage (reading R2) for block b: rows above
  // row 0 / below row H - 1 and columns outside the image take the nearest
  // image pixel's bit (prev: the stage's word of block b - 1).  A unit starts
  // at row 0 or at a row >= 16 (its start is a multiple of the unit height,
  // itself a multiple of 16, past the view's first row, which is 0 or >= 64),
  // so a block that reaches above row 0 starts at row -3 or lies wholly above
  // the image, where it feeds no output.
  __device__ __forceinline__ uint32_t replicate(int64_t b, uint32_t m, uint32_t prev) {
    const int64_t r0 = Y0 - 3 + 16 * b;  // image row of bit-row 0
    if (r0 < 0) {  // top: rows -3..-1 take row 0 (bit-row 3)
      const uint32_t pr = (m >> 24) & 0x3u;
      m = (m & 0x03FFFFFFu) | (pr << 26) | (pr << 28) | (pr << 30);
    }
    if (r0 + 15 >= H) {  // bottom: rows >= H take row H - 1
      const int64_t rH = H - 1 - r0;
      if (rH >= 0) {
        const uint32_t keep = 0xFFFFFFFFu << (2 * (15 - rH));
        const uint32_t pr = (m >> (30 - 2 * rH)) & 0x3u;
        m = (m & keep) | ((pr * 0x55555555u) & ~keep);
      } else {
        m = (prev & 0x3u) * 0x55555555u;
      }
    }
    if (border) m = fix_cols_bits(m);
    return m;
  }

  // Hybrid median with window k (3 or 5) of block own (prev / next: the blocks
  // above / below).
  __device__ __forceinline__ uint32_t median(uint32_t prev, uint32_t own, uint32_t next, int k) {
    const uint32_t oP = __shfl_up_sync(kFull, own, 1), oX = __shfl_down_sync(kFull, own, 1);
    const uint32_t pP = __shfl_up_sync(kFull, prev, 1), pX = __shfl_down_sync(kFull, prev, 1);
    const uint32_t xP = __shfl_up_sync(kFull, next, 1), xX = __shfl_down_sync(kFull, next, 1);
    const uint32_t E1o = e1(own, oX), W1o = w1(own, oP), E1p = e1(prev, pX), W1p = w1(prev, pP);
    const uint32_t E1n = e1(next, xX), W1n = w1(next, xP);
    if (k == 5) {  // two columns over: the neighbour lane's word itself
      const uint32_t plus[9] = {own, E1o, W1o, oX, oP, n1(own, prev), s1(own, next), n2(own, prev), s2(own, next)};
      const uint32_t cross[9] = {own, n1(E1o, E1p), n1(W1o, W1p), s1(E1o, E1n), s1(W1o, W1n),
                                 n2(oX, pX), n2(oP, pP), s2(oX, xX), s2(oP, xP)};
      return maj3(maj9(plus), maj9(cross), own);
    }
    if (k == 7) {  // three columns over: the neighbour lane's one-column shifts
      const uint32_t E3o = __shfl_down_sync(kFull, E1o, 1), W3o = __shfl_up_sync(kFull, W1o, 1);
      const uint32_t E3p = __shfl_down_sync(kFull, E1p, 1), W3p = __shfl_up_sync(kFull, W1p, 1);
      const uint32_t E3n = __shfl_down_sync(kFull, E1n, 1), W3n = __shfl_up_sync(kFull, W1n, 1);
      const uint32_t plus[13] = {own, E1o, W1o, oX, oP, E3o, W3o, n1(own, prev), s1(own, next),
                                 n2(own, prev), s2(own, next), n3(own, prev), s3(own, next)};
      const uint32_t cross[13] = {own, n1(E1o, E1p), n1(W1o, W1p), s1(E1o, E1n), s1(W1o, W1n),
                                  n2(oX, pX), n2(oP, pP), s2(oX, xX), s2(oP, xP),
                                  n3(E3o, E3p), n3(W3o, W3p), s3(E3o, E3n), s3(W3o, W3n)};
      return maj3(maj13(plus), maj13(cross), own);
    }
    const uint32_t plus[5] = {own, E1o, W1o, n1(own, prev), s1(own, next)};
    const uint32_t cross[5] = {own, n1(E1o, E1p), n1(W1o, W1p), s1(E1o, E1n), s1(W1o, W1n)};
    return maj3(maj5(plus), maj5(cross), own);
  }

  // Store of the output rows of block b (mask words h).
  __device__ __forceinline__ void store(int64_t b, uint32_t h) {
    const int64_t x = xs + 2 * lane;
    const bool lane_out = lane >= kLeftHalo / 2 && lane < (kLeftHalo + kOutCols) / 2 && x < W;
    if (!lane_out) return;
    const int64_t ybase = Y0 - 3 + 16 * b;
    // rows [ybase + rlo, ybase + rhi) of this block belong to the unit
    const int64_t lo64 = Y0 - ybase, hi64 = Y1 - ybase;
    const int rlo = lo64 < 0 ? 0 : static_cast<int>(lo64), rhi = hi64 > 16 ? 16 : static_cast<int>(hi64);
    if (rhi <= rlo) return;
    const uint32_t rows = ((1u << rhi) - 1u) & ~((1u << rlo) - 1u);
    uint8_t *dst = v.out + (ybase - v.y_begin) * v.out_pitch + x;
    const uint32_t op = static_cast<uint32_t>(v.out_pitch);
    // FX_CHECKED: the rows written lie in the view's output rows, the columns in the image
    if (!FX_GUARD(x >= 0 && x < W && ybase + rlo >= v.y_begin && ybase + rhi <= v.y_end)) return;
    if (vstore && x + 1 < W) {
      // two rows at a time: their 4 bits (h bits 28-2r .. 31-2r) spread to 4
      // bytes by one multiply, then one 16-bit store per row
#pragma unroll
      for (int r = 0; r < 16; r += 2) {
        const uint32_t q = (h >> (28 - 2 * r)) & 0xFu;
        const uint32_t e = (q * 0x00204081u) & 0x01010101u;  // bit k of q -> byte k
        if (rows & (1u << r)) *reinterpret_cast<uint16_t *>(dst + static_cast<uint64_t>(r) * op) = static_cast<uint16_t>(e >> 16);
        if (rows & (2u << r))
          *reinterpret_cast<uint16_t *>(dst + static_cast<uint64_t>(r + 1) * op) = static_cast<uint16_t>(e);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (!(rows & (1u << r))) continue;
        const uint32_t pr = (h >> (30 - 2 * r)) & 0x3u;
        uint8_t *d = dst + static_cast<uint64_t>(r) * op;
        d[0] = static_cast<uint8_t>(pr & 1u);
        if (x + 1 < W) d[1] = static_cast<uint8_t>(pr >> 1);
      }
    }
  }

  // End of the 16 steps of group g: block g is packed in acc_.
  __device__ __forceinline__ bool end_group(int64_t g) {
    if (checking()) {
      if (__any_sync(kFull, tracked_max() > static_cast<uint32_t>(kp.fbound))) return false;
    }
    uint32_t m = 0;
    int64_t gm;  // block index of m (the mask M)
    if constexpr (kSrcZ) {
      // crossings of block g - 1 (a replicated stage), then the standard
      // deviation over them, extraction and OR for block g - 2
      gm = g - 2;
      uint32_t z[2] = {0, 0};
#pragma unroll
      for (int f = 0; f < 2; ++f)
        if (g >= 0) z[f] = replicate(g - 1, crossings(f), sw_[kZA + f][lane]);
      if (g >= 1) {  // from block -1 on: wide median lists reach the rows above the unit
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const uint32_t za = sw_[kZA + f][lane];
          m |= za & ~sw_[kPcf + f][lane] & sd_over_z(sw_[kZB + f][lane], za, z[f], f);
        }
        m = replicate(gm, m, sw_[kMA][lane]);
      }
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        sw_[kZB + f][lane] = sw_[kZA + f][lane];
        sw_[kZA + f][lane] = z[f];
        sw_[kPcf + f][lane] = blk(5 * f + 4);
      }
    } else {
      gm = g - 1;
      if (g >= 0) m = mask_block(g - 1);  // from block -1 on: wide median lists reach the rows above the unit
    }
    // Median levels (Sec. 3.4, repeated per Sec. 4.2): level l + 1 of block
    // gm - l - 1 from level l of blocks gm - l - 2 .. gm - l; every level but
    // the last is a replicated stage (reading R2).  Without a median the mask
    // of block gm - 1 is stored (the same one block of delay).
    const int nl = nhmf();
    uint32_t cur = m;
    if (kRm <= kCompactRm || nl <= 1) {  // a single level (or none) without the level loop
      const uint32_t a = sw_[kLev][lane];
      // compact strips: the one level is a window-3 median
      if (gm >= 1) store(gm - 1, nl ? median(sw_[kLev + 1][lane], a, m, kRm <= kCompactRm ? 3 : hmf_at(0)) : a);
      sw_[kLev + 1][lane] = a;
      sw_[kLev][lane] = m;
    } else {
#pragma unroll 1
      for (int l = 0; l < nl; ++l) {
        const uint32_t a = sw_[kLev + 2 * l][lane], b = sw_[kLev + 2 * l + 1][lane];
        sw_[kLev + 2 * l + 1][lane] = a;
        sw_[kLev + 2 * l][lane] = cur;
        const uint32_t h = median(b, a, cur, hmf_at(l));
        if (!FX_GUARD(l < FX_MAX_HMF_LEVELS && kLev + 2 * l + 2 <= kZA)) break;
        cur = l + 1 < nl ? replicate(gm - l - 1, h, sw_[kLev + 2 * l + 2][lane]) : h;
      }
      if (gm - nl >= 0) store(gm - nl, cur);  // the last level's words of block gm - nl
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      sw_[kPneg + f][lane] = blk(5 * f);
      sw_[kPpos + f][lane] = blk(5 * f + 1);
      sw_[kPsS + f][lane] = blk(5 * f + 3);
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) blk(i) = acc_[i];
    return true;
  }

  template <bool kChk>
  __device__ __forceinline__ void four_steps(int32_t t0) {  // t0 = 4k relative to Y0
    step<0, kChk>(t0);
    step<1, kChk>(t0 + 1);
    step<2, kChk>(t0 + 2);
    step<3, kChk>(t0 + 3);
  }

  // kTail: skip the steps past the last row any output needs (single-image
  // launches; the batched kernels, whose units are long, run without it).
  template <bool kTail = true>
  __device__ bool run() {
    // Rows Y0-8 .. Y0-1 (k = -2, -1; from Y0-12 for wide strips) fill the rings;
    // they compute the rows above the unit that its outputs depend on (the mask
    // rows down to Y0 - r_m).  Bit blocks span 16 rows (four
    // iterations); block b covers rows [Y0 - 3 + 16b, Y0 + 13 + 16b) and its
    // median is stored at the end of group b + 2.
    if constexpr (kAsync) {
      // rows 4 kK0 .. 4 kK0 + 6 into their slots (slot of row t = t & 7); each
      // step refills the slot read one step before with the row seven ahead
#pragma unroll
      for (int i = 0; i < kRingRows - 1; ++i) load_row_async(ring_h_ + 128u * ((4 * kK0 + i) & 7), 4 * kK0 + i);
    } else {
      load_row<0>(4 * kK0);
      load_row<1>(4 * kK0 + 1);
      load_row<2>(4 * kK0 + 2);
      load_row<3>(4 * kK0 + 3);
    }
    const uint32_t ring0 = ring_h_;
    const int32_t bmax = static_cast<int32_t>((Y1 - Y0 + 2) / 16);
    // one more block of delay per extra median level and for the crossing-map source
    const int32_t iters = 4 * (bmax + 2 + (nhmf() > 1 ? nhmf() : 1) + (kSrcZ ? 1 : 0));
    // the last step whose row feeds an output: the bits of row r are packed at
    // step r + 3, and the last output row needs the median radius, its south
    // neighbour (+1) and, for the crossing-map source, the deviation's 2 rows
    [[maybe_unused]] const int32_t t_end = static_cast<int32_t>(Y1 - Y0 - 1) + kp.r_m + 4 + (kSrcZ ? 2 : 0);
    for (int32_t k = kK0; k < iters; ++k) {
      if constexpr (kTail) {
        if (4 * k > t_end) {
          // past the rows any output needs: keep the bit positions of the block
          // schedule (four steps of two columns) without computing the steps
#pragma unroll
          for (int i = 0; i < 12; ++i) acc_[i] <<= 8;
          if ((k & 3) == 3 && !end_group(k >> 2)) {
            async_drain();
            return false;
          }
          continue;
        }
      }
      // centre rows of this iteration: 4k - 2 .. 4k + 1 and loaded rows 4k + la ..
      // 4k + 3 + la (relative to Y0; la = the load distance); the fix-ups act only
      // on a border strip, at image row 0 and past row H - 1, and loads clamp only
      // outside [rlo, rhi].  The unchecked body loads without clamping, so it may
      // run only when every row it loads lies in [rlo, rhi].
      constexpr int32_t la = kAsync ? kRingRows - 1 : 4;
      const bool chk = border || (4 * k - 2 <= -Y0rel && -Y0rel <= 4 * k + 1) || 4 * k + 1 >= Hrel ||
                       4 * k + la < rlo || 4 * k + 3 + la > rhi;
      if constexpr (kAsync) {
        // ring slots of this iteration's rows 4k .. 4k + 3: 4 (k & 1) + S
        ring_h_ = ring0 + ((k & 1) ? 512u : 0u);
        ring_o_ = ring0 + ((k & 1) ? 0u : 512u);
      }
      if (chk) four_steps<true>(4 * k);
      else four_steps<false>(4 * k);
      if ((k & 3) == 3 && !end_group(k >> 2)) {
        async_drain();
        return false;
      }
    }
    async_drain();
    return true;
  }
};

}  // namespace st

// Work units: output columns [52 ux, 52 ux + 52), rows [y_begin + uh uy,
// + uh) of the view, computed by the calling warp.
//
// fast_unit runs the FP32 path.  A strip that meets a value above
// KParams::fbound stops before storing anything that depends on it and marks
// its first output byte with kRedo (masks are otherwise 0 or 1);
// fast_unit_redo, launched afterwards on the same stream, recomputes exactly
// the marked strips on the integer path (every strip when fbound < 0).  The
// two paths are separate kernels so the rare integer path does not raise the
// register allocation of the FP32 one.
constexpr uint8_t kRedo = 0xFF;

__device__ __forceinline__ uint8_t *unit_marker(const ImageView &v, int64_t ux, int64_t uy, int uh, int uw) {
  return v.out + (uy * uh) * v.out_pitch + ux * uw;
}

// Per-warp shared words of the streaming path (the caller's kernel owns one
// array of this type per CTA and passes the warp's slice).
constexpr int kStripWords = 48;  // 32 block words + two 8-row input rings
using StripWords = uint32_t[kWarpsPerCta][kStripWords][32];
__device__ __forceinline__ uint32_t (*warp_words(StripWords &w))[32] { return w[(threadIdx.x >> 5) % kWarpsPerCta]; }

// kF32Log selects the FP32-LoG mode (KParams::f32log) at compile time; kSd2 =
// !KParams::sd_same (kSd2 = true is correct for any thresholds); kSrcZ =
// (KParams::source == 1); kRm = the strip class.
template <typename T, bool kF32Log, bool kPair, bool kSd2, bool kSrcZ, bool kTail = true, int kRm = kNarrowRm,
          class Cst = RuntimeConsts>
__device__ __forceinline__ void fast_unit(const ImageView &v, const KParams &kp, int64_t ux, int64_t uy, int,
                                          int uh, uint32_t (*words)[32]) {
  constexpr int kMode = kF32Log ? st::kModeF32Log : st::kModeF32;
  using S = st::Strip<T, kMode, kPair, kSd2, kSrcZ, kRm, Cst>;
  static_assert(S::kWords + 2 * S::kRingRows == kStripWords, "shared word layout");
  if (kp.fbound < 0) return;
  constexpr int uw = strip_width(kSrcZ, kRm);
  const int64_t X0 = ux * uw;
  const int64_t Y0 = v.y_begin + uy * uh;
  const int64_t Y1 = Y0 + uh < v.y_end ? Y0 + uh : v.y_end;
  S s(v, kp, X0, Y0, Y1, words);
  if (!s.template run<kTail>() && (threadIdx.x & 31) == 0 &&
      FX_GUARD(uy * uh < v.y_end - v.y_begin && ux * uw < v.width))
    *unit_marker(v, ux, uy, uh, uw) = kRedo;
}

// The streaming first pass of fx_extract: one unit per warp, units in
// row-band order (unit = CTA * kWarpsPerCta + warp; ux = unit % units_x),
// kFirstPassCtas CTAs per SM.
template <typename T, bool kF32Log, bool kPair, bool kSd2, bool kSrcZ, int kRm, class Cst>
__global__ void __launch_bounds__(32 * kWarpsPerCta, kFirstPassCtas)
    stream_kernel(const __grid_constant__ ImageView v, const __grid_constant__ KParams kp, int64_t units_x,
                  int64_t units, int uh) {
  __shared__ StripWords words;
  const int64_t unit = static_cast<int64_t>(blockIdx.x) * kWarpsPerCta + (threadIdx.x >> 5);
  if (unit >= units) return;  // whole warps only
  fast_unit<T, kF32Log, kPair, kSd2, kSrcZ, true, kRm, Cst>(v, kp, unit % units_x, unit / units_x, 0, uh,
                                                           warp_words(words));
}

template <typename T, bool kF32Log, bool kSrcZ, int kRm = kNarrowRm>
__device__ __forceinline__ void fast_unit_redo(const ImageView &v, const KParams &kp, int64_t ux, int64_t uy,
                                               int, int uh, uint32_t (*words)[32]) {
  constexpr int kMode = kF32Log ? st::kModeF32LogWide : st::kModeInt;
  constexpr int uw = strip_width(kSrcZ, kRm);
  if (kp.fbound >= 0) {
    uint8_t mark = 0;
    if ((threadIdx.x & 31) == 0 && FX_GUARD(uy * uh < v.y_end - v.y_begin && ux * uw < v.width))
      mark = *unit_marker(v, ux, uy, uh, uw);
    if (__shfl_sync(st::kFull, mark, 0) != kRedo) return;
  }
  const int64_t X0 = ux * uw;
  const int64_t Y0 = v.y_begin + uy * uh;
  const int64_t Y1 = Y0 + uh < v.y_end ? Y0 + uh : v.y_end;
  st::Strip<T, kMode, false, true, kSrcZ, kRm> s(v, kp, X0, Y0, Y1, words);
  s.run();
}

}  // namespace fx
