// fx_hmf.cu -- the hybrid median filter (Sec. 3.4) on uint8 / uint16 images.
//
// Output = median(median of the '+' subgroup, median of the 'x' subgroup,
// centre), the subgroups being the centre row/column segment and the two
// diagonals of the k x k window (2k - 1 values each, k = 3, 5 or 7); pixels
// outside the image take the value of the nearest image pixel (replicated
// borders).  Medians come from exact min/max identities:
//   med3(a, b, c)  = max(min(a, b), min(max(a, b), c))
//   med5           = med3(c, max(min(a, b), min(d, e)), min(max(a, b), max(d, e)))
//   med9 of three triples = med3(max of the triples' minima,
//                                med3 of their medians, min of their maxima)
// and, for the 13 values of a window-7 subgroup, forgetful selection: of any
// m + 1 values of a set of 2m - 1, the smallest and the largest lie on either
// side of the set's median, so dropping both keeps the median of the rest;
// hold 8 values, drop the two ends, take in the next value, and repeat until
// three values are left, whose median is the answer.  The ends are found by
// compare-exchanges (min and max), which keep every other value.
//
// One warp walks down a strip of 60 output columns (56 for k = 7: a
// 64-column window with one halo lane, two for k = 7, on each side), one
// input row per step.  Lane l holds the two pixels of window columns 2l,
// 2l+1 as one u16x2 word, so every min/max handles two pixels.  A ring of k
// rows keeps, per row, the words of the lane's pixels shifted by -k/2..k/2
// columns (neighbour lanes by shuffle, one-column shifts by byte selection);
// loads are issued k rows ahead into a ring of their own and never sit inside
// a branch.  For uint16 images read as
// aligned pairs the loads go instead through a per-warp shared-memory ring of
// kAsyncRows rows filled by cp.async, kAsyncRows - 1 rows ahead: many more
// bytes in flight per SM than a register ring allows, at no register cost.
#include <cstdint>
#include <utility>

#include "fx_checked.cuh"
#include "fx_internal.h"

namespace fx {
namespace {

constexpr int kHmfUnitH = 128; // output rows per strip unit
constexpr int kHmfWarps = 4;   // warps per CTA
constexpr int kAsyncRows = 16; // depth of the shared-memory load ring (power of two)
constexpr unsigned kAll = 0xffffffffu;

// 4-byte asynchronous copy global -> shared (the thread's own group queue)
__device__ __forceinline__ void cp_async4(uint32_t *dst, const void *src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t vmin(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t vmax(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t med3(uint32_t a, uint32_t b, uint32_t c) {
  return vmax(vmin(a, b), vmin(vmax(a, b), c));
}
__device__ __forceinline__ uint32_t med5(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e) {
  return med3(c, vmax(vmin(a, b), vmin(d, e)), vmin(vmax(a, b), vmax(d, e)));
}
// minimum, median and maximum of a triple
__device__ __forceinline__ void sort3(uint32_t a, uint32_t b, uint32_t c, uint32_t &lo, uint32_t &md,
                                      uint32_t &hi) {
  const uint32_t mn = vmin(a, b), mx = vmax(a, b);
  lo = vmin(mn, c);
  hi = vmax(mx, c);
  md = vmax(mn, vmin(mx, c));
}
// median of {a0..a2} U {b0..b2} U {c0..c2}
__device__ __forceinline__ uint32_t med9(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t b0, uint32_t b1,
                                         uint32_t b2, uint32_t c0, uint32_t c1, uint32_t c2) {
  uint32_t al, am, ah, bl, bm, bh, cl, cm, ch;
  sort3(a0, a1, a2, al, am, ah);
  sort3(b0, b1, b2, bl, bm, bh);
  sort3(c0, c1, c2, cl, cm, ch);
  return med3(vmax(vmax(al, bl), cl), med3(am, bm, cm), vmin(vmin(ah, bh), ch));
}
// compare-exchange: a <- min, b <- max
__device__ __forceinline__ void cx(uint32_t &a, uint32_t &b) {
  const uint32_t lo = vmin(a, b);
  b = vmax(a, b);
  a = lo;
}
// the minimum of v[0..N-1] to v[0], the maximum to v[N-1], the other values
// kept in v[1..N-2]: order each pair (0, 1), (2, 3), ..., then run the pairs'
// smaller values (and an unpaired last one) through v[0] and their larger
// values through v[N-1]
template <int N>
__device__ __forceinline__ void ends(uint32_t (&v)[8]) {
#pragma unroll
  for (int i = 0; i + 1 < N; i += 2) cx(v[i], v[i + 1]);
#pragma unroll
  for (int i = 2; i < N; i += 2) cx(v[0], v[i]);
#pragma unroll
  for (int i = 1; i < N - 1; i += 2) cx(v[i], v[N - 1]);
}
// median of 13 values by forgetful selection (v: the first 8, x: the other 5)
__device__ __forceinline__ uint32_t med13(uint32_t (&v)[8], const uint32_t (&x)[5]) {
  ends<8>(v);  // keep v[1..6]
  v[0] = x[0];
  ends<7>(v);  // keep v[1..5]
  v[0] = x[1];
  ends<6>(v);  // keep v[1..4]
  v[0] = x[2];
  ends<5>(v);  // keep v[1..3]
  v[0] = x[3];
  ends<4>(v);  // keep v[1..2]
  return med3(v[1], v[2], x[4]);
}

// kPair: one aligned load of the lane's two pixels per row (base and pitch
// multiples of two pixels, even width), the clamped columns picked by a byte
// selector at use; otherwise two single-pixel loads at the clamped columns.
template <typename T, int K, bool kPair>
struct HmfStrip {
  static constexpr int R = K / 2;
  static constexpr int kHalo = (R + 1) / 2;     // halo lanes on each side
  static constexpr int kOut = 64 - 4 * kHalo;   // output columns per strip
  static constexpr int L = K;  // loads run one window (k rows) ahead
  // aligned uint16 pairs: 4-byte asynchronous copies into the warp's ring
  static constexpr bool kAsync = kPair && sizeof(T) == 2;
  uint32_t (*ring_)[32] = nullptr;  // kAsyncRows x 32 words of this warp (kAsync)
  const unsigned char *p0_, *p1_;  // this lane's load addresses in image row 0
  uint32_t sel_;
  int64_t pitch, H, Y0, Y1, W, x;
  unsigned char *out_;
  int64_t opitch;
  int lane;
  // 32-bit row arithmetic: step t reads input row Y0 - R + clamp(t, tlo_, thi_)
  // at q0_ / q1_ + (clamped t - tb_) * pitch, and writes output row Y0 + t - 2R
  // (when in [0, nrows_)) at outb_ + (t - 2R) * opitch
  int32_t tlo_, thi_, tb_, nrows_;
  const unsigned char *q0_, *q1_;
  unsigned char *outb_;
  uint32_t pitch32_, opitch32_;
  bool vst_;  // one store of the lane's two output pixels (aligned rows)
  bool colok_;  // FX_CHECKED: this lane's loaded columns lie in the image
  uint32_t raw0_[L], raw1_[L];  // loaded pixels of the next L rows
  uint32_t win_[K][K];          // per ring row: the pair words shifted by -R..R columns (index d + R)

  __device__ HmfStrip(const T *img, int64_t W_, int64_t H_, int64_t pitch_, T *out, int64_t opitch_, int64_t X0,
                      int64_t Y0_, int64_t Y1_)
      : pitch(pitch_), H(H_), Y0(Y0_), Y1(Y1_), W(W_), out_(reinterpret_cast<unsigned char *>(out)),
        opitch(opitch_) {
    lane = threadIdx.x & 31;
    x = X0 - 2 * kHalo + 2 * lane;
    const int64_t c0 = x < 0 ? 0 : (x >= W ? W - 1 : x), c1 = x + 1 < 0 ? 0 : (x + 1 >= W ? W - 1 : x + 1);
    if constexpr (kPair) {
      const int64_t cb = (c0 < W - 2 ? c0 : W - 2) & ~int64_t{1};  // even pair holding both columns
      p0_ = p1_ = reinterpret_cast<const unsigned char *>(img) + cb * static_cast<int64_t>(sizeof(T));
      colok_ = cb >= 0 && cb + 1 < W;
      const uint32_t h0 = static_cast<uint32_t>(c0 - cb), h1 = static_cast<uint32_t>(c1 - cb);
      if constexpr (sizeof(T) == 2) sel_ = (h0 ? 0x32u : 0x10u) | ((h1 ? 0x32u : 0x10u) << 8);
      else sel_ = h0 | 0x40u | (h1 << 8) | 0x4000u;
    } else {
      p0_ = reinterpret_cast<const unsigned char *>(img) + c0 * static_cast<int64_t>(sizeof(T));
      p1_ = reinterpret_cast<const unsigned char *>(img) + c1 * static_cast<int64_t>(sizeof(T));
      colok_ = c0 >= 0 && c0 < W && c1 >= 0 && c1 < W;
      sel_ = 0x5410u;
    }
    // pitches are below 2^32 bytes and sides below 2^30 (checked by the host)
    tlo_ = static_cast<int32_t>(R - Y0);
    thi_ = static_cast<int32_t>(H - 1 - Y0 + R);
    tb_ = tlo_ > 0 ? tlo_ : 0;
    q0_ = p0_ + (Y0 - R + tb_) * pitch;
    q1_ = p1_ + (Y0 - R + tb_) * pitch;
    pitch32_ = static_cast<uint32_t>(pitch);
    opitch32_ = static_cast<uint32_t>(opitch);
    nrows_ = static_cast<int32_t>(Y1 - Y0);
    outb_ = out_ + Y0 * opitch + x * static_cast<int64_t>(sizeof(T));
    vst_ = reinterpret_cast<uintptr_t>(out_) % (2 * sizeof(T)) == 0 && opitch % (2 * sizeof(T)) == 0;
  }

  // byte offset of the input row that step t reads (clamped to the image)
  __device__ __forceinline__ uint64_t row_off(int32_t t) const {
    const int32_t tc = t < tlo_ ? tlo_ : (t > thi_ ? thi_ : t);
    return static_cast<uint64_t>(static_cast<uint32_t>(tc - tb_)) * pitch32_;
  }

  // kAsync: input row Y0 - R + t (clamped) into ring slot t mod kAsyncRows, as
  // one commit group
  __device__ __forceinline__ void issue(int32_t t) {
    const int32_t tc = t < tlo_ ? tlo_ : (t > thi_ ? thi_ : t);  // the row row_off reads
    if (FX_GUARD(colok_ && tc >= tb_ && Y0 - R + tc < H)) cp_async4(&ring_[t & (kAsyncRows - 1)][lane], q0_ + row_off(t));
    cp_async_commit();
  }

  // input row Y0 - R + t (clamped to the image) into load slot S
  template <int S>
  __device__ __forceinline__ void load(int32_t t) {
    const uint64_t off = row_off(t);
    const int32_t tc = t < tlo_ ? tlo_ : (t > thi_ ? thi_ : t);
    if (!FX_GUARD(colok_ && tc >= tb_ && Y0 - R + tc < H)) return;
    if constexpr (kPair) {
      if constexpr (sizeof(T) == 2) raw0_[S] = __ldg(reinterpret_cast<const uint32_t *>(q0_ + off));
      else raw0_[S] = __ldg(reinterpret_cast<const uint16_t *>(q0_ + off));
    } else {
      raw0_[S] = __ldg(reinterpret_cast<const T *>(q0_ + off));
      raw1_[S] = __ldg(reinterpret_cast<const T *>(q1_ + off));
    }
  }

  template <int SL>
  __device__ __forceinline__ void step(int32_t t) {  // SL = t % L; window slot S = t % K
    constexpr int S = SL % K;
    // (column 2l, 2l+1) as a u16x2 word; the selection also copies the slot before it is refilled
    uint32_t w;
    if constexpr (kAsync) {
      cp_async_wait<kAsyncRows - 2>();  // row t has landed (rows t + 1 .. t + kAsyncRows - 2 may be in flight)
      w = __byte_perm(ring_[t & (kAsyncRows - 1)][lane], 0, sel_);
    } else {
      w = kPair ? __byte_perm(raw0_[SL], 0, sel_) : __byte_perm(raw0_[SL], raw1_[SL], 0x5410);
      load<SL>(t + L);
    }
    const uint32_t pv = __shfl_up_sync(kAll, w, 1), nx = __shfl_down_sync(kAll, w, 1);
    // refill the slot of row t - 1, whose value the previous step has used
    if constexpr (kAsync) issue(t + kAsyncRows - 1);
    uint32_t *row = win_[S];
    if constexpr (R == 3) {
      const uint32_t pv2 = __shfl_up_sync(kAll, w, 2), nx2 = __shfl_down_sync(kAll, w, 2);
      row[0] = __byte_perm(pv2, pv, 0x5432);  // columns -3, -2
      row[6] = __byte_perm(nx, nx2, 0x5432);  //  3, 4
    }
    if constexpr (R >= 2) {
      row[R - 2] = pv;  // -2, -1
      row[R + 2] = nx;  //  2, 3
    }
    row[R - 1] = __byte_perm(pv, w, 0x5432);  // -1, 0
    row[R] = w;
    row[R + 1] = __byte_perm(w, nx, 0x5432);  //  1, 2
    // centre row t - R of the window rows t - 2R .. t (ring slot (S + K - i) % K holds row t - i)
    const int32_t orow = t - 2 * R;  // output row relative to Y0
    if (orow < 0 || orow >= nrows_) return;
    constexpr int c = (S + K - R) % K;
    const uint32_t *C = win_[c];
    uint32_t h;
    if constexpr (K == 7) {
      const uint32_t *N3 = win_[(S + 1) % K], *N2 = win_[(S + 2) % K], *N1 = win_[(S + 3) % K];
      const uint32_t *S1 = win_[(S + 5) % K], *S2 = win_[(S + 6) % K], *S3 = win_[S];
      // '+': the centre row segment and the column; 'x': both diagonals
      uint32_t plus8[8] = {C[0], C[1], C[2], C[3], C[4], C[5], C[6], N3[3]};
      const uint32_t plus5[5] = {N2[3], N1[3], S1[3], S2[3], S3[3]};
      uint32_t cross8[8] = {N3[0], N2[1], N1[2], C[3], S1[4], S2[5], S3[6], N3[6]};
      const uint32_t cross5[5] = {N2[5], N1[4], S1[2], S2[1], S3[0]};
      h = med3(med13(plus8, plus5), med13(cross8, cross5), C[3]);
    } else if constexpr (K == 5) {
      const uint32_t *N2 = win_[(S + 1) % K], *N1 = win_[(S + 2) % K], *S1 = win_[(S + 4) % K], *S2 = win_[S];
      const uint32_t plus = med9(C[0], C[1], C[2], C[3], C[4], N2[2], N1[2], S1[2], S2[2]);
      const uint32_t cross = med9(N2[0], N1[1], C[2], S1[3], S2[4], N2[4], N1[3], S1[1], S2[0]);
      h = med3(plus, cross, C[2]);
    } else {
      const uint32_t *N1 = win_[(S + 1) % K], *S1 = win_[S];
      const uint32_t plus = med5(C[0], N1[1], C[1], S1[1], C[2]);
      const uint32_t cross = med5(N1[0], N1[2], C[1], S1[0], S1[2]);
      h = med3(plus, cross, C[1]);
    }
    if (lane < kHalo || lane > 31 - kHalo || x >= W) return;
    if (!FX_GUARD(x >= 0 && Y0 + orow < H)) return;
    unsigned char *d = outb_ + static_cast<uint64_t>(static_cast<uint32_t>(orow)) * opitch32_;
    if (vst_ && x + 1 < W) {  // x is even, so the pair is aligned
      if constexpr (sizeof(T) == 2) *reinterpret_cast<uint32_t *>(d) = h;
      else *reinterpret_cast<uint16_t *>(d) = static_cast<uint16_t>((h & 0xFFu) | ((h >> 8) & 0xFF00u));
    } else {
      *reinterpret_cast<T *>(d) = static_cast<T>(h & 0xFFFFu);
      if (x + 1 < W) *reinterpret_cast<T *>(d + sizeof(T)) = static_cast<T>(h >> 16);
    }
  }

  template <int... S>
  __device__ __forceinline__ void steps(int32_t t0, std::integer_sequence<int, S...>) {
    (step<S>(t0 + S), ...);
  }
  template <int... S>
  __device__ __forceinline__ void loads(std::integer_sequence<int, S...>) {
    (load<S>(S), ...);
  }

  __device__ void run() {
    if constexpr (kAsync) {
      for (int t = 0; t < kAsyncRows - 1; ++t) issue(t);
    } else {
      loads(std::make_integer_sequence<int, L>{});
    }
    const int32_t last = nrows_ + 2 * R;  // steps 0 .. last - 1 cover output rows Y0 .. Y1 - 1
    for (int32_t t0 = 0; t0 < last; t0 += L) steps(t0, std::make_integer_sequence<int, L>{});
    if constexpr (kAsync) cp_async_wait<0>();  // no copy outlives the warp
  }
};

template <typename T, int K, bool kPair>
__global__ void __launch_bounds__(32 * kHmfWarps) hmf_stream_kernel(const T *img, int64_t W, int64_t H,
                                                                     int64_t pitch, T *out, int64_t out_pitch,
                                                                     int64_t units_x, int64_t units) {
  const int64_t unit = static_cast<int64_t>(blockIdx.x) * kHmfWarps + (threadIdx.x >> 5);
  if (unit >= units) return;  // whole warps only
  const int64_t ux = unit % units_x, uy = unit / units_x;
  const int64_t Y0 = uy * kHmfUnitH, Y1 = Y0 + kHmfUnitH < H ? Y0 + kHmfUnitH : H;
  HmfStrip<T, K, kPair> s(img, W, H, pitch, out, out_pitch, ux * HmfStrip<T, K, kPair>::kOut, Y0, Y1);
  if constexpr (HmfStrip<T, K, kPair>::kAsync) {
    __shared__ uint32_t ring[kHmfWarps][kAsyncRows][32];
    s.ring_ = ring[threadIdx.x >> 5];
  }
  s.run();
}

template <typename T>
cudaError_t launch_hmf(const T *img, int64_t W, int64_t H, int64_t pitch, T *out, int64_t opitch, int k,
                       cudaStream_t s) {
  const int64_t out_w = HmfStrip<T, 3, true>::kOut;  // the same for k = 3 and 5
  const int64_t uw = k == 7 ? HmfStrip<T, 7, true>::kOut : out_w;
  const int64_t units_x = (W + uw - 1) / uw, units = units_x * ((H + kHmfUnitH - 1) / kHmfUnitH);
  const int64_t blocks = (units + kHmfWarps - 1) / kHmfWarps;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned g = static_cast<unsigned>(blocks);
  constexpr int nt = 32 * kHmfWarps;
  const int64_t two = 2 * static_cast<int64_t>(sizeof(T));
  const bool pair = reinterpret_cast<uintptr_t>(img) % two == 0 && pitch % two == 0 && W % 2 == 0;
  if (k == 7) {
    if (pair) hmf_stream_kernel<T, 7, true><<<g, nt, 0, s>>>(img, W, H, pitch, out, opitch, units_x, units);
    else hmf_stream_kernel<T, 7, false><<<g, nt, 0, s>>>(img, W, H, pitch, out, opitch, units_x, units);
  } else if (k == 5) {
    if (pair) hmf_stream_kernel<T, 5, true><<<g, nt, 0, s>>>(img, W, H, pitch, out, opitch, units_x, units);
    else hmf_stream_kernel<T, 5, false><<<g, nt, 0, s>>>(img, W, H, pitch, out, opitch, units_x, units);
  } else {
    if (pair) hmf_stream_kernel<T, 3, true><<<g, nt, 0, s>>>(img, W, H, pitch, out, opitch, units_x, units);
    else hmf_stream_kernel<T, 3, false><<<g, nt, 0, s>>>(img, W, H, pitch, out, opitch, units_x, units);
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace fx

using namespace fx;

extern "C" fx_status fx_hybrid_median(const void *img, int64_t width, int64_t height, int64_t pitch_bytes,
                                      fx_dtype dtype, int32_t window, void *out, int64_t out_pitch_bytes,
                                      void *stream) {
  NvtxRange range("fx_hybrid_median");
  if (window != 3 && window != 5 && window != 7) return FX_ERR_INVALID_ARG;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e =
      dtype == FX_U8 ? launch_hmf(static_cast<const uint8_t *>(img), width, height, pitch_bytes,
                                  static_cast<uint8_t *>(out), out_pitch_bytes, window, s)
                     : launch_hmf(static_cast<const uint16_t *>(img), width, height, pitch_bytes,
                                  static_cast<uint16_t *>(out), out_pitch_bytes, window, s);
  return e == cudaSuccess ? FX_OK : FX_ERR_CUDA;
}

namespace fx {
FX_CHECK_COUNTER(checked_count_hmf)
}  // namespace fx
