/*
 * fx_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU oracle for the automated feature extraction of
 * "GPU Accelerated Automated Feature Extraction from Satellite Images"
 * (Tejaswi, Rao, Nair, Prasad; arXiv 1304.3992).  Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg load it; the
 * product library never links, imports or executes it, and it shares no
 * code, header or table with the CUDA path.
 *
 * Every stage is one full pass over a full-width array, in the order of
 * Sec. 4.1: two LoG convolutions (Eq. 1) -> zero crossings on each response
 * plus the contrast threshold (Sec. 3.2) -> the local standard-deviation
 * test (Eq. 2, Sec. 4.1) -> OR-combination of the two extracted maps
 * (Sec. 4.1) -> hybrid median filter (Sec. 3.4), optionally repeated with
 * several window sizes (Sec. 4, Sec. 4.2).
 *
 * All quantities are integers below 2^53 (in the FP32-LoG mode, R9:
 * multiples of 2^-14 below 2^40), so FP64 evaluates every stage exactly; no
 * tolerance is involved anywhere in the oracle.
 *
 * Readings of the paper where it is silent or garbled (numbers as in the
 * design notes):
 *   R1  sigma = 0.5 and 20 (Sec. 4.1 says "variance"; Eq. 1 is in sigma).
 *       Eq. 1 sampled on the 5x5 grid is not zero-sum, so the mask is
 *       mean-subtracted, scaled to max |w| = Q, rounded half away from zero,
 *       and the centre is reset to minus the sum of the other 24 weights.
 *   R2  Borders: every stage array extends outside the image by
 *       replication, S(x,y) := S(clamp(x,y)) (Sec. 4.1 gives pad sizes only).
 *   R3  Zero crossing (Sec. 3.2): a pixel with L != 0 is a crossing iff it
 *       has an opposite-signed 4-neighbour and its |L| is smaller than the
 *       |L| of every opposite-signed 4-neighbour, an exact tie going to the
 *       negative pixel (for integer L this is key(v) = 2|v| + [v > 0]
 *       compared strictly); a pixel with L == 0 is a crossing iff
 *       L(W)L(E) < 0 or L(N)L(S) < 0.  The contrast
 *       max - min of L over the pixel and its 4 neighbours must exceed
 *       t_zc (strict).
 *   R4  Standard deviation (Eq. 2): unbiased s over the 5x5 window centred
 *       on the pixel (Lambda = 25); if s5 > t_sdmax the decision is
 *       s3 > t_sd3 over the 3x3 window (Lambda = 9), else s5 > t_sd5.
 *       s > T is evaluated exactly as D > (T*T)*Lambda*(Lambda-1) with
 *       D = Lambda*sum(a^2) - (sum a)^2 (for T < 0 the test always passes).
 *       The values a are the image (source 0) or the binary zero-crossing
 *       map of the same branch (source 1).
 *   R5  The two extracted maps are OR-combined.
 *   R6  Hybrid median with window k (3, 5 or 7; Sec. 3.4 leaves the size to
 *       the application): the '+' subgroup is the centre row and column
 *       segment (2k-1 pixels), the 'x' subgroup the two diagonals (2k-1
 *       pixels); output = median(med+, medx, centre).  A list of windows
 *       applies the filter repeatedly, in order (Sec. 4, Sec. 4.2).
 *   R7  Output is a uint8 image of 0/1.
 *   R9  FP32-LoG mode (log_mode 1, non-integer masks): the mean-removed
 *       samples of R1, scaled to max |w| = Q, are rounded half away from zero
 *       to multiples of g = 2^(e-23), 2^e the smallest power of two >= Q,
 *       and the centre is reset to minus the exact sum of the other 24.  The
 *       oracle applies these masks exactly; the library's FP32 evaluation may
 *       differ only where a decision is within rounding of its threshold.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Parameter vector layout (all doubles), see oracle/__init__.py. */
enum {
  P_SIGMA1 = 0, P_SIGMA2, P_Q, P_TZC1, P_TZC2, P_TSD5_1, P_TSD5_2,
  P_TSDMAX_1, P_TSDMAX_2, P_TSD3_1, P_TSD3_2, P_SOURCE,
  P_HMF0, P_HMF1, P_HMF2, P_HMF3, P_LOGMODE, P_COUNT
};

#define ORACLE_MAX_HMF 4

/* Status codes returned to the Python wrapper. */
enum { O_OK = 0, O_BAD_ARG = 1, O_NOMEM = 2, O_INTERNAL = 3 };

static long long clampll(long long v, long long lo, long long hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

/* ---------------------------------------------------------------- Eq. 1 */

/* LoG(x,y) of Eq. 1 (Sec. 3.1). */
static double log_eq1(double sigma, double x, double y) {
  double r2 = x * x + y * y;
  double s2 = sigma * sigma;
  return -1.0 / (M_PI * s2 * s2) * (1.0 - r2 / (2.0 * s2)) * exp(-r2 / (2.0 * s2));
}

static double round_half_away(double v) {
  return v >= 0.0 ? floor(v + 0.5) : -floor(-v + 0.5);
}

/* Reading R1: Eq. 1 sampled on x, y in {-2..2}, made zero-sum and integer.
 * g receives the raw samples, w the integer mask (row-major, w[(dy+2)*5+dx+2]). */
int fxo_log_mask(double sigma, double q, double *g, double *w) {
  if (!(sigma > 0.0) || !isfinite(sigma) || !(q >= 1.0) || !isfinite(q)) return O_BAD_ARG;
  double samp[25], mean = 0.0;
  for (int dy = -2; dy <= 2; ++dy)
    for (int dx = -2; dx <= 2; ++dx) {
      samp[(dy + 2) * 5 + (dx + 2)] = log_eq1(sigma, dx, dy);
      mean += samp[(dy + 2) * 5 + (dx + 2)];
    }
  mean /= 25.0;
  double maxabs = 0.0;
  for (int i = 0; i < 25; ++i) {
    double c = fabs(samp[i] - mean);
    if (c > maxabs) maxabs = c;
  }
  if (!(maxabs > 0.0)) return O_BAD_ARG;
  double others = 0.0;
  for (int i = 0; i < 25; ++i) {
    w[i] = round_half_away(q * (samp[i] - mean) / maxabs);
    if (i != 12) others += w[i];
  }
  w[12] = -others;
  if (g)
    for (int i = 0; i < 25; ++i) g[i] = samp[i];
  return O_OK;
}

/* Reading R9: the same centred samples on the grid g = 2^(e-23) (every
 * weight then fits the 24-bit FP32 significand), centre reset to keep the
 * mask exactly zero-sum.  w receives the weights as doubles (exact). */
int fxo_log_mask_fp32(double sigma, double q, double *w) {
  if (!(sigma > 0.0) || !isfinite(sigma) || !(q >= 1.0) || !(q <= 1048576.0)) return O_BAD_ARG;
  double samp[25], mean = 0.0;
  for (int dy = -2; dy <= 2; ++dy)
    for (int dx = -2; dx <= 2; ++dx) {
      samp[(dy + 2) * 5 + (dx + 2)] = log_eq1(sigma, dx, dy);
      mean += samp[(dy + 2) * 5 + (dx + 2)];
    }
  mean /= 25.0;
  double maxabs = 0.0;
  for (int i = 0; i < 25; ++i) {
    double c = fabs(samp[i] - mean);
    if (c > maxabs) maxabs = c;
  }
  if (!(maxabs > 0.0)) return O_BAD_ARG;
  int e = 0;
  while (ldexp(1.0, e) < q) ++e;
  double grid = ldexp(1.0, e - 23), others = 0.0;
  for (int i = 0; i < 25; ++i) {
    w[i] = round_half_away(q * (samp[i] - mean) / maxabs / grid) * grid;
    if (i != 12) others += w[i];
  }
  w[12] = -others;
  return O_OK;
}

/* ------------------------------------------------------------- planes */

/* A full-width stage array holding image rows [y_lo, y_hi).  Reads go through
 * clamp(x, y) (reading R2), so a stage extends outside the image by
 * replication of its own border values. */
typedef struct {
  double *v;
  long long W, H, y_lo, y_hi;
  int bad; /* set when a clamped read falls outside [y_lo, y_hi) */
} plane;

static int plane_init(plane *p, long long W, long long H, long long y_lo, long long y_hi) {
  p->W = W; p->H = H; p->y_lo = y_lo; p->y_hi = y_hi; p->bad = 0;
  const long long n = (y_hi > y_lo ? y_hi - y_lo : 0) * (W > 0 ? W : 0);
  p->v = (double *)calloc(n > 0 ? (size_t)n : 1, sizeof(double));
  return p->v ? O_OK : O_NOMEM;
}

static double plane_at(plane *p, long long x, long long y) {
  long long xc = clampll(x, 0, p->W - 1), yc = clampll(y, 0, p->H - 1);
  if (yc < p->y_lo || yc >= p->y_hi) { p->bad = 1; return 0.0; }
  return p->v[(yc - p->y_lo) * p->W + xc];
}

static void plane_set(plane *p, long long x, long long y, double val) {
  p->v[(y - p->y_lo) * p->W + x] = val;
}

typedef struct {
  const uint8_t *base;
  int elem;            /* 1 = uint8, 2 = uint16 */
  long long W, H, pitch; /* pitch in bytes */
} image;

/* The input image with replicated borders (reading R2). */
static double pix(const image *im, long long x, long long y) {
  long long xc = clampll(x, 0, im->W - 1), yc = clampll(y, 0, im->H - 1);
  const uint8_t *row = im->base + yc * im->pitch;
  if (im->elem == 1) return (double)row[xc];
  uint16_t v;
  memcpy(&v, row + 2 * xc, 2);
  return (double)v;
}

/* ------------------------------------------------------------ stages */

/* Sec. 4.1: the 5x5 LoG mask applied to every pixel's 5x5 neighbourhood. */
static void stage_log(const image *im, const double *w, plane *L) {
  for (long long y = L->y_lo; y < L->y_hi; ++y)
    for (long long x = 0; x < im->W; ++x) {
      double acc = 0.0;
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx)
          acc += w[(dy + 2) * 5 + (dx + 2)] * pix(im, x + dx, y + dy);
      plane_set(L, x, y, acc);
    }
}

/* Reading R3: v (non-zero, opposite in sign to q) has the smaller magnitude;
 * an exact tie goes to the negative pixel. */
static int smaller_than(double v, double q) {
  return fabs(v) < fabs(q) || (fabs(v) == fabs(q) && v < 0.0);
}

/* Sec. 3.2 with reading R3: zero crossing of L at every pixel of Z. */
static void stage_zero_crossing(plane *L, plane *Z) {
  for (long long y = Z->y_lo; y < Z->y_hi; ++y)
    for (long long x = 0; x < Z->W; ++x) {
      double v = plane_at(L, x, y);
      double nb[4] = {plane_at(L, x - 1, y), plane_at(L, x + 1, y),
                      plane_at(L, x, y - 1), plane_at(L, x, y + 1)}; /* W E N S */
      int z;
      if (v != 0.0) {
        int any = 0, smallest = 1;
        for (int k = 0; k < 4; ++k)
          if (v * nb[k] < 0.0) {
            any = 1;
            if (!smaller_than(v, nb[k])) smallest = 0;
          }
        z = any && smallest;
      } else {
        z = (nb[0] * nb[1] < 0.0) || (nb[2] * nb[3] < 0.0);
      }
      plane_set(Z, x, y, z ? 1.0 : 0.0);
    }
}

/* Sec. 3.2: keep crossings whose positive maximum minus negative minimum over
 * the pixel and its 4 neighbours is large: max - min > t_zc. */
static void stage_contrast(plane *L, double t_zc, plane *C) {
  for (long long y = C->y_lo; y < C->y_hi; ++y)
    for (long long x = 0; x < C->W; ++x) {
      double v[5] = {plane_at(L, x, y), plane_at(L, x - 1, y), plane_at(L, x + 1, y),
                     plane_at(L, x, y - 1), plane_at(L, x, y + 1)};
      double mx = v[0], mn = v[0];
      for (int k = 1; k < 5; ++k) {
        if (v[k] > mx) mx = v[k];
        if (v[k] < mn) mn = v[k];
      }
      plane_set(C, x, y, (mx - mn > t_zc) ? 1.0 : 0.0);
    }
}

/* Eq. 2 exactly: s > T  <=>  Lambda*sum(a^2) - (sum a)^2 > T^2*Lambda*(Lambda-1). */
static int sd_exceeds(double sum, double sumsq, double lambda, double T) {
  if (T < 0.0) return 1;
  double D = lambda * sumsq - sum * sum;
  return D > ((T * T) * lambda) * (lambda - 1.0);
}

/* Sec. 4.1 with reading R4: the 5x5 standard deviation, re-computed on the
 * 3x3 neighbourhood when it exceeds the maximum threshold. */
static void stage_stddev(const image *im, plane *Zsrc, int source, double t5, double tmax,
                         double t3, plane *S) {
  for (long long y = S->y_lo; y < S->y_hi; ++y)
    for (long long x = 0; x < S->W; ++x) {
      double s5 = 0, q5 = 0, s3 = 0, q3 = 0;
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          double a = source == 0 ? pix(im, x + dx, y + dy) : plane_at(Zsrc, x + dx, y + dy);
          s5 += a; q5 += a * a;
          if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) { s3 += a; q3 += a * a; }
        }
      int keep;
      if (sd_exceeds(s5, q5, 25.0, tmax)) keep = sd_exceeds(s3, q3, 9.0, t3);
      else keep = sd_exceeds(s5, q5, 25.0, t5);
      plane_set(S, x, y, keep ? 1.0 : 0.0);
    }
}

static double median_of(double *v, int n) { /* insertion sort, then middle */
  for (int i = 1; i < n; ++i) {
    double t = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
    v[j + 1] = t;
  }
  return v[(n - 1) / 2];
}

/* Sec. 3.4 with reading R6: hybrid median of window k at every pixel of O. */
static void stage_hmf(plane *M, int k, plane *O) {
  int r = k / 2;
  double plus[13], cross[13], three[3]; /* 2k - 1 <= 13 */
  for (long long y = O->y_lo; y < O->y_hi; ++y)
    for (long long x = 0; x < O->W; ++x) {
      int np = 0, nc = 0;
      for (int d = -r; d <= r; ++d) {
        plus[np++] = plane_at(M, x + d, y);
        if (d != 0) plus[np++] = plane_at(M, x, y + d);
        cross[nc++] = plane_at(M, x + d, y + d);
        if (d != 0) cross[nc++] = plane_at(M, x + d, y - d);
      }
      three[0] = median_of(plus, np);
      three[1] = median_of(cross, nc);
      three[2] = plane_at(M, x, y);
      plane_set(O, x, y, median_of(three, 3));
    }
}

/* ----------------------------------------------------------- driver */

static int row_window(plane *p, long long W, long long H, long long y0, long long y1, long long r) {
  return plane_init(p, W, H, clampll(y0 - r, 0, H), clampll(y1 + r, 0, H));
}

/*
 * Compute output rows [y0, y1) of the extraction of an image.
 *   img    first byte of image row 0; rows are pitch bytes apart
 *   elem   1 (uint8) or 2 (uint16)
 *   prm    P_COUNT doubles (layout above); hmf windows 0 mark unused slots
 *   out    (y1-y0) x W bytes, row-major, receives 0/1
 *   stages optional: NULL, or 9 planes of (y1-y0) x W doubles receiving
 *          L1, L2, Z1, Z2, C1, C2, S1, S2, M for the same rows
 */
int fxo_extract(const void *img, int elem, long long W, long long H, long long pitch,
                const double *prm, int nprm, long long y0, long long y1, uint8_t *out,
                double *stages) {
  if (!img || !out || !prm || nprm != P_COUNT) return O_BAD_ARG;
  if (elem != 1 && elem != 2) return O_BAD_ARG;
  if (W < 1 || H < 1 || pitch < W * elem || y0 < 0 || y1 > H || y0 >= y1) return O_BAD_ARG;
  int source = (int)prm[P_SOURCE];
  if (source != 0 && source != 1) return O_BAD_ARG;
  int hmf[ORACLE_MAX_HMF], nh = 0, r_m = 0;
  for (int i = 0; i < ORACLE_MAX_HMF; ++i) {
    int k = (int)prm[P_HMF0 + i];
    if (k == 0) break;
    if (k != 3 && k != 5 && k != 7) return O_BAD_ARG;
    hmf[nh++] = k;
    r_m += k / 2;
  }
  for (int i = 0; i < P_COUNT; ++i)
    if (isnan(prm[i])) return O_BAD_ARG;

  int log_mode = (int)prm[P_LOGMODE];
  if (log_mode != 0 && log_mode != 1) return O_BAD_ARG;
  image im = {(const uint8_t *)img, elem, W, H, pitch};
  double w[2][25];
  for (int f = 0; f < 2; ++f) {
    int rc0 = log_mode == 0 ? fxo_log_mask(prm[P_SIGMA1 + f], prm[P_Q], NULL, w[f])
                            : fxo_log_mask_fp32(prm[P_SIGMA1 + f], prm[P_Q], w[f]);
    if (rc0 != O_OK) return O_BAD_ARG;
  }

  /* Rows each stage needs so that the output rows are complete. */
  long long r_s = r_m;                      /* S, C, Z(as used), E, M */
  long long r_z = r_s + (source == 1 ? 2 : 0);
  long long r_l = r_z + 1;

  plane L[2], Z[2], C[2], S[2], M, tmp[2];
  memset(L, 0, sizeof L); memset(Z, 0, sizeof Z); memset(C, 0, sizeof C);
  memset(S, 0, sizeof S); memset(&M, 0, sizeof M); memset(tmp, 0, sizeof tmp);
  int rc = O_OK, bad = 0;
  for (int f = 0; f < 2 && rc == O_OK; ++f) {
    if ((rc = row_window(&L[f], W, H, y0, y1, r_l)) != O_OK) break;
    if ((rc = row_window(&Z[f], W, H, y0, y1, r_z)) != O_OK) break;
    if ((rc = row_window(&C[f], W, H, y0, y1, r_s)) != O_OK) break;
    if ((rc = row_window(&S[f], W, H, y0, y1, r_s)) != O_OK) break;
    stage_log(&im, w[f], &L[f]);
    stage_zero_crossing(&L[f], &Z[f]);
    stage_contrast(&L[f], prm[P_TZC1 + f], &C[f]);
    stage_stddev(&im, &Z[f], source, prm[P_TSD5_1 + f], prm[P_TSDMAX_1 + f],
                 prm[P_TSD3_1 + f], &S[f]);
  }
  if (rc == O_OK) rc = row_window(&M, W, H, y0, y1, r_m);
  if (rc == O_OK) {
    /* Sec. 4.1: extracted map per branch = crossing AND contrast AND stddev;
     * the two maps are combined (reading R5: OR). */
    for (long long y = M.y_lo; y < M.y_hi; ++y)
      for (long long x = 0; x < W; ++x) {
        int m = 0;
        for (int f = 0; f < 2; ++f)
          if (plane_at(&Z[f], x, y) != 0.0 && plane_at(&C[f], x, y) != 0.0 &&
              plane_at(&S[f], x, y) != 0.0)
            m = 1;
        plane_set(&M, x, y, m ? 1.0 : 0.0);
      }
    /* Sec. 3.4 / Sec. 4.2: the hybrid median, once per listed window. */
    plane *cur = &M;
    long long r_left = r_m;
    for (int i = 0; i < nh && rc == O_OK; ++i) {
      r_left -= hmf[i] / 2;
      plane *nxt = &tmp[i & 1];
      free(nxt->v);
      if ((rc = row_window(nxt, W, H, y0, y1, r_left)) != O_OK) break;
      stage_hmf(cur, hmf[i], nxt);
      bad |= cur->bad;
      cur = nxt;
    }
    if (rc == O_OK) {
      for (long long y = y0; y < y1; ++y)
        for (long long x = 0; x < W; ++x)
          out[(y - y0) * W + x] = plane_at(cur, x, y) != 0.0 ? 1 : 0;
      bad |= cur->bad;
    }
    if (rc == O_OK && stages) {
      long long n = (y1 - y0) * W;
      plane *src[9] = {&L[0], &L[1], &Z[0], &Z[1], &C[0], &C[1], &S[0], &S[1], &M};
      for (int s = 0; s < 9; ++s)
        for (long long y = y0; y < y1; ++y)
          for (long long x = 0; x < W; ++x)
            stages[s * n + (y - y0) * W + x] = plane_at(src[s], x, y);
    }
  }
  for (int f = 0; f < 2; ++f) {
    bad |= L[f].bad | Z[f].bad | C[f].bad | S[f].bad;
    free(L[f].v); free(Z[f].v); free(C[f].v); free(S[f].v);
  }
  bad |= M.bad;
  free(M.v); free(tmp[0].v); free(tmp[1].v);
  if (rc == O_OK && bad) rc = O_INTERNAL;
  return rc;
}

/* Sec. 3.4 on its own: the hybrid median (reading R6, one window) of a
 * uint8/uint16 image, the grayscale form of the filter. */
int fxo_hybrid_median(const void *img, int elem, long long W, long long H, long long pitch,
                      int k, uint16_t *out) {
  if (!img || !out || (elem != 1 && elem != 2) || W < 1 || H < 1 || pitch < W * elem) return O_BAD_ARG;
  if (k != 3 && k != 5 && k != 7) return O_BAD_ARG;
  image im = {(const uint8_t *)img, elem, W, H, pitch};
  plane P, O;
  if (plane_init(&P, W, H, 0, H) != O_OK) return O_NOMEM;
  if (plane_init(&O, W, H, 0, H) != O_OK) { free(P.v); return O_NOMEM; }
  for (long long y = 0; y < H; ++y)
    for (long long x = 0; x < W; ++x) plane_set(&P, x, y, pix(&im, x, y));
  stage_hmf(&P, k, &O);
  for (long long i = 0; i < W * H; ++i) out[i] = (uint16_t)O.v[i];
  free(P.v); free(O.v);
  return O_OK;
}
