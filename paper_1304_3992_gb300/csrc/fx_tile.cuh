// fx_tile.cuh -- the general fused extraction tile (device code).
//
//
// One CTA computes a TW x TH tile of the output mask.  It stages its input
// tile plus the full input halo in shared memory once, then evaluates every
// stage of Sec. 4.1 on chip, one shared-memory array per stage:
//   LoG x2 (Eq. 1) -> zero crossing x2 (Sec. 3.2) -> contrast, standard
//   deviation (Eq. 2) and OR-combination -> hybrid median passes (Sec. 3.4).
// Each stage array covers the tile plus the radius the later stages still
// need, and every entry holds the stage's value at the CLAMPED image
// coordinate, which realises replicated borders for every stage.
//
// This kernel handles every parameter combination (any number of median
// passes, either standard-deviation source, any dtype) in exact integer
// arithmetic, or with FP32 responses in the FP32-LoG mode.  The streaming
// kernel in fx_stream.cu is the fast path for every configuration whose median
// radii add up to at most 3; both must agree bit for bit in either mode (the
// allocation-free entry point always runs this kernel).
#include <cstdint>

#pragma once
#include "fx_checked.cuh"
#include "fx_internal.h"

namespace fx {
namespace gen {

constexpr int TW = 64;
constexpr int TH = 32;
constexpr int NT = 256;

__device__ __forceinline__ int64_t clampll(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

struct Radii {
  int m, z, l, i;
};

__host__ __device__ inline Radii radii_of(const KParams &kp) {
  Radii r;
  r.m = kp.r_m;
  r.z = r.m + (kp.source == 1 ? 2 : 0);
  r.l = r.z + 1;
  r.i = r.l + 2;
  return r;
}

__host__ __device__ inline int area(int r) { return (TW + 2 * r) * (TH + 2 * r); }

inline size_t general_smem_bytes(const KParams &kp) {
  Radii r = radii_of(kp);
  size_t b = 0;
  b += sizeof(int32_t) * area(r.i);
  b += sizeof(int32_t) * 2 * area(r.l);
  b += 2 * area(r.z);
  b += 2 * area(r.m);
  return b;
}

// A stage array over the tile expanded by radius r.  ox, oy are the image
// coordinates of its element (0, 0).
template <typename V>
struct Arr {
  V *p;
  int64_t ox, oy;
  int w, h;  // columns and rows
  __device__ V &at_clamped(int64_t xc, int64_t yc) const {  // xc, yc already clamped
    int64_t i = (yc - oy) * w + (xc - ox);
    if (!FX_GUARD(yc - oy >= 0 && yc - oy < h && xc - ox >= 0 && xc - ox < w)) i = 0;
    return p[i];
  }
};

template <typename T>
__device__ __forceinline__ int32_t load_px(const ImageView &v, int64_t x, int64_t y) {
  if (!FX_GUARD(y >= v.row0 && y < v.row_lim && x >= 0 && x < v.width)) return 0;
  const uint8_t *row = static_cast<const uint8_t *>(v.img) + (y - v.row0) * v.pitch;
  return static_cast<int32_t>(reinterpret_cast<const T *>(row)[x]);
}

__device__ __forceinline__ int64_t zc_key(int64_t v) { return 2 * (v < 0 ? -v : v) + (v > 0 ? 1 : 0); }

__device__ __forceinline__ bool opposite(int64_t a, int64_t b) { return (a < 0 && b > 0) || (a > 0 && b < 0); }

// FP32-LoG mode (KParams::f32log): L is stored as float bits in the same arrays.
__device__ __forceinline__ bool opposite_f(float a, float b) { return (a < 0.f && b > 0.f) || (a > 0.f && b < 0.f); }
// c beats an opposite-signed q: smaller magnitude, ties to the negative pixel (reading R3)
__device__ __forceinline__ bool beats_f(float c, float q) {
  return fabsf(c) < fabsf(q) || (fabsf(c) == fabsf(q) && c < 0.f);
}

// Ring index (squared radius 0, 1, 2, 4, 5, 8 -> 0..5) of the offset (dx, dy).
__device__ __forceinline__ int ring_index(int dx, int dy) {
  const int r2 = dx * dx + dy * dy;
  return r2 == 0 ? 0 : r2 == 1 ? 1 : r2 == 2 ? 2 : r2 == 4 ? 3 : r2 == 5 ? 4 : 5;
}

// FP32-LoG response from exact ring sums: the operations of the streaming
// kernel, in its order (d_c = R_c - n_c R0, products added left to right).
__device__ __forceinline__ float log_f32(const KParams &kp, int f, const int32_t R[6]) {
  const float d1 = static_cast<float>(R[1] - 4 * R[0]), d2 = static_cast<float>(R[2] - 4 * R[0]);
  const float d4 = static_cast<float>(R[3] - 4 * R[0]), d5 = static_cast<float>(R[4] - 8 * R[0]);
  const float d8 = static_cast<float>(R[5] - 4 * R[0]);
  float l = __fmaf_rn(kp.ringf[f][1], d1, 0.0f);  // from +0: never -0
  l = __fmaf_rn(kp.ringf[f][2], d2, l);
  l = __fmaf_rn(kp.ringf[f][3], d4, l);
  l = __fmaf_rn(kp.ringf[f][4], d5, l);
  return __fmaf_rn(kp.ringf[f][5], d8, l);
}

// Contrast test of Sec. 3.2 over the pixel and its 4 neighbours (clamped
// coordinates): max - min > t_zc, or fl(max - min) > tzf in the FP32-LoG mode.
__device__ __forceinline__ bool contrast_pass(const KParams &kp, int f, const Arr<int32_t> &L, int64_t xc, int64_t yc,
                                              int64_t xw, int64_t xe, int64_t yn, int64_t ys) {
  const int32_t v[5] = {L.at_clamped(xc, yc), L.at_clamped(xw, yc), L.at_clamped(xe, yc), L.at_clamped(xc, yn),
                        L.at_clamped(xc, ys)};
  if (kp.f32log) {
    float mx = __int_as_float(v[0]), mn = mx;
    for (int k = 1; k < 5; ++k) {
      mx = fmaxf(mx, __int_as_float(v[k]));
      mn = fminf(mn, __int_as_float(v[k]));
    }
    return __fsub_rn(mx, mn) > kp.tzf[f];
  }
  int32_t mx = v[0], mn = v[0];
  for (int k = 1; k < 5; ++k) {
    mx = max(mx, v[k]);
    mn = min(mn, v[k]);
  }
  return mx - mn > kp.tzc[f];
}

// One TW x TH output tile whose top-left output pixel is (x0, y0).  All NT
// threads of the CTA must call it; smem holds general_smem_bytes(kp) bytes.
template <typename T>
__device__ void general_tile(const ImageView &v, const KParams &kp, int64_t x0, int64_t y0,
                             unsigned char *smem) {
  const Radii R = radii_of(kp);
  const int64_t W = v.width, H = v.height;

  unsigned char *cur = smem;
  Arr<int32_t> I{reinterpret_cast<int32_t *>(cur), x0 - R.i, y0 - R.i, TW + 2 * R.i, TH + 2 * R.i};
  cur += sizeof(int32_t) * area(R.i);
  Arr<int32_t> L[2];
  for (int f = 0; f < 2; ++f) {
    L[f] = Arr<int32_t>{reinterpret_cast<int32_t *>(cur), x0 - R.l, y0 - R.l, TW + 2 * R.l, TH + 2 * R.l};
    cur += sizeof(int32_t) * area(R.l);
  }
  Arr<uint8_t> Z[2];
  for (int f = 0; f < 2; ++f) {
    Z[f] = Arr<uint8_t>{cur, x0 - R.z, y0 - R.z, TW + 2 * R.z, TH + 2 * R.z};
    cur += area(R.z);
  }
  Arr<uint8_t> M[2];
  for (int k = 0; k < 2; ++k) {
    M[k] = Arr<uint8_t>{cur, x0 - R.m, y0 - R.m, TW + 2 * R.m, TH + 2 * R.m};
    cur += area(R.m);
  }

  // a1: one read of the input tile plus halo, clamped to the image.
  for (int i = threadIdx.x; i < area(R.i); i += NT) {
    int64_t x = clampll(I.ox + i % I.w, 0, W - 1), y = clampll(I.oy + i / I.w, 0, H - 1);
    if (FX_GUARD(i < I.w * I.h)) I.p[i] = load_px<T>(v, x, y);
  }
  __syncthreads();

  // a2: the two LoG responses (Eq. 1 masks on the 5x5 neighbourhood).
  for (int i = threadIdx.x; i < area(R.l); i += NT) {
    int64_t xc = clampll(L[0].ox + i % L[0].w, 0, W - 1), yc = clampll(L[0].oy + i / L[0].w, 0, H - 1);
    if (kp.f32log) {
      int32_t R[6] = {0, 0, 0, 0, 0, 0};  // exact ring sums (< 2^20)
      for (int dy = -2; dy <= 2; ++dy) {
        int64_t yy = clampll(yc + dy, 0, H - 1);
        for (int dx = -2; dx <= 2; ++dx) R[ring_index(dx, dy)] += I.at_clamped(clampll(xc + dx, 0, W - 1), yy);
      }
      if (FX_GUARD(i < L[0].w * L[0].h)) {
        L[0].p[i] = __float_as_int(log_f32(kp, 0, R));
        L[1].p[i] = __float_as_int(log_f32(kp, 1, R));
      }
      continue;
    }
    int32_t acc0 = 0, acc1 = 0;
    for (int dy = -2; dy <= 2; ++dy) {
      int64_t yy = clampll(yc + dy, 0, H - 1);
      for (int dx = -2; dx <= 2; ++dx) {
        int32_t a = I.at_clamped(clampll(xc + dx, 0, W - 1), yy);
        acc0 += kp.w[0][(dy + 2) * 5 + dx + 2] * a;
        acc1 += kp.w[1][(dy + 2) * 5 + dx + 2] * a;
      }
    }
    if (FX_GUARD(i < L[0].w * L[0].h)) {
      L[0].p[i] = acc0;
      L[1].p[i] = acc1;
    }
  }
  __syncthreads();

  // a3: zero crossings among the 4 neighbours (Sec. 3.2).
  for (int i = threadIdx.x; i < area(R.z); i += NT) {
    int64_t xc = clampll(Z[0].ox + i % Z[0].w, 0, W - 1), yc = clampll(Z[0].oy + i / Z[0].w, 0, H - 1);
    int64_t xw = clampll(xc - 1, 0, W - 1), xe = clampll(xc + 1, 0, W - 1);
    int64_t yn = clampll(yc - 1, 0, H - 1), ys = clampll(yc + 1, 0, H - 1);
    for (int f = 0; f < 2; ++f) {
      if (kp.f32log) {
        const float c = __int_as_float(L[f].at_clamped(xc, yc));
        const float nb[4] = {__int_as_float(L[f].at_clamped(xw, yc)), __int_as_float(L[f].at_clamped(xe, yc)),
                             __int_as_float(L[f].at_clamped(xc, yn)), __int_as_float(L[f].at_clamped(xc, ys))};
        bool z;
        if (c != 0.f) {
          bool any = false, smallest = true;
          for (int k = 0; k < 4; ++k)
            if (opposite_f(c, nb[k])) {
              any = true;
              if (!beats_f(c, nb[k])) smallest = false;
            }
          z = any && smallest;
        } else {
          z = opposite_f(nb[0], nb[1]) || opposite_f(nb[2], nb[3]);
        }
        if (FX_GUARD(i < Z[f].w * Z[f].h)) Z[f].p[i] = z;
        continue;
      }
      int64_t c = L[f].at_clamped(xc, yc);
      int64_t nb[4] = {L[f].at_clamped(xw, yc), L[f].at_clamped(xe, yc), L[f].at_clamped(xc, yn),
                       L[f].at_clamped(xc, ys)};
      bool z;
      if (c != 0) {
        bool any = false, smallest = true;
        for (int k = 0; k < 4; ++k)
          if (opposite(c, nb[k])) {
            any = true;
            if (!(zc_key(c) < zc_key(nb[k]))) smallest = false;
          }
        z = any && smallest;
      } else {
        z = opposite(nb[0], nb[1]) || opposite(nb[2], nb[3]);
      }
      if (FX_GUARD(i < Z[f].w * Z[f].h)) Z[f].p[i] = z;
    }
  }
  __syncthreads();

  // a4-a6: contrast, standard deviation (Eq. 2), extraction and OR-combination.
  for (int i = threadIdx.x; i < area(R.m); i += NT) {
    int64_t xc = clampll(M[0].ox + i % M[0].w, 0, W - 1), yc = clampll(M[0].oy + i / M[0].w, 0, H - 1);
    int64_t xw = clampll(xc - 1, 0, W - 1), xe = clampll(xc + 1, 0, W - 1);
    int64_t yn = clampll(yc - 1, 0, H - 1), ys = clampll(yc + 1, 0, H - 1);
    bool m = false;
    // image-source sums are shared by both branches
    int64_t s5 = 0, q5 = 0, s3 = 0, q3 = 0;
    if (kp.source == 0) {
      for (int dy = -2; dy <= 2; ++dy) {
        int64_t yy = clampll(yc + dy, 0, H - 1);
        for (int dx = -2; dx <= 2; ++dx) {
          int64_t a = I.at_clamped(clampll(xc + dx, 0, W - 1), yy);
          s5 += a;
          q5 += a * a;
          if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
            s3 += a;
            q3 += a * a;
          }
        }
      }
    }
    for (int f = 0; f < 2; ++f) {
      if (!Z[f].at_clamped(xc, yc)) continue;
      if (!contrast_pass(kp, f, L[f], xc, yc, xw, xe, yn, ys)) continue;
      if (kp.source == 1) {
        s5 = q5 = s3 = q3 = 0;
        for (int dy = -2; dy <= 2; ++dy) {
          int64_t yy = clampll(yc + dy, 0, H - 1);
          for (int dx = -2; dx <= 2; ++dx) {
            int64_t a = Z[f].at_clamped(clampll(xc + dx, 0, W - 1), yy);
            s5 += a;
            q5 += a;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
              s3 += a;
              q3 += a;
            }
          }
        }
      }
      int64_t d5 = 25 * q5 - s5 * s5, d3 = 9 * q3 - s3 * s3;
      bool keep = (d5 > kp.tsdmax[f]) ? (d3 > kp.tsd3[f]) : (d5 > kp.tsd5[f]);
      if (keep) m = true;
    }
    if (FX_GUARD(i < M[0].w * M[0].h)) M[0].p[i] = m;
  }
  __syncthreads();

  // a7: hybrid median passes (Sec. 3.4) on the binary map; binary median = majority.
  int src = 0;
  int r_cur = R.m;
  Arr<uint8_t> in = M[0];
  for (int lev = 0; lev < kp.nhmf; ++lev) {
    const int k = kp.hmf[lev], r = k / 2, r_out = r_cur - r;
    Arr<uint8_t> out{M[src ^ 1].p, x0 - r_out, y0 - r_out, TW + 2 * r_out, TH + 2 * r_out};
    for (int i = threadIdx.x; i < area(r_out); i += NT) {
      int64_t xc = clampll(out.ox + i % out.w, 0, W - 1), yc = clampll(out.oy + i / out.w, 0, H - 1);
      int plus = 0, cross = 0;
      for (int d = -r; d <= r; ++d) {
        int64_t xd = clampll(xc + d, 0, W - 1), yd = clampll(yc + d, 0, H - 1), ym = clampll(yc - d, 0, H - 1);
        plus += in.at_clamped(xd, yc);
        cross += in.at_clamped(xd, yd);
        if (d != 0) {
          plus += in.at_clamped(xc, yd);
          cross += in.at_clamped(xd, ym);
        }
      }
      int c = in.at_clamped(xc, yc);
      int mp = plus > r * 2, mxv = cross > r * 2;  // majority of 2k-1 = 4r+1 values
      if (FX_GUARD(i < out.w * out.h)) out.p[i] = (mp + mxv + c) >= 2;
    }
    __syncthreads();
    src ^= 1;
    r_cur = r_out;
    in = out;
  }

  // a8: one write of the mask tile.
  for (int i = threadIdx.x; i < TW * TH; i += NT) {
    int64_t x = x0 + i % TW, y = y0 + i / TW;
    if (x < W && y < v.y_end && FX_GUARD(x >= 0 && y >= v.y_begin))
      v.out[(y - v.y_begin) * v.out_pitch + x] = M[src].p[(i / TW) * TW + i % TW];
  }
}


}  // namespace gen
}  // namespace fx
