"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test names the passage it follows.  Together they are chosen so that a
plausible slip anywhere in the oracle (a dropped term, a wrong sign or index,
a transposed operand, a wrong tie rule, an off-by-one window) fails one of
them: closed forms of Eq. 1, mask invariants, the step-edge closed forms of
the LoG / zero crossing / Eq. 2, library medians for the hybrid median,
library standard deviations for Eq. 2, symmetry and invariance properties of
the whole pipeline, and an independent pure-Python brute force on tiny
images.
"""
import itertools
import math
import statistics

import numpy as np
import pytest

import oracle
from oracle import brute
from gen import scenes


def params(**kw):
    p = oracle.default_params(1.0)
    p.update(kw)
    return p


# ------------------------------------------------------------------ Eq. 1

def test_eq1_samples_match_closed_forms():
    """Sec. 3.1, Eq. 1 at sigma = 0.5: LoG(0,0) = -16/pi, LoG(1,0) = (16/pi) e^-2,
    LoG(1,1) = (16/pi) 3 e^-4, LoG(2,0) = (16/pi) 7 e^-8; at sigma = 20:
    LoG(0,0) = -1/(pi 20^4)."""
    g, _ = oracle.log_mask(0.5)
    k = 16 / math.pi
    assert g[2, 2] == pytest.approx(-k, rel=1e-14)
    assert g[2, 3] == pytest.approx(k * math.exp(-2), rel=1e-14)
    assert g[1, 3] == pytest.approx(3 * k * math.exp(-4), rel=1e-14)
    assert g[2, 4] == pytest.approx(7 * k * math.exp(-8), rel=1e-14)
    assert g[0, 2] == pytest.approx(7 * k * math.exp(-8), rel=1e-14)
    g20, _ = oracle.log_mask(20.0)
    assert g20[2, 2] == pytest.approx(-1 / (math.pi * 20.0 ** 4), rel=1e-14)
    # raw Eq. 1 samples are not zero-sum on the 5x5 grid (the reason for reading R1)
    assert g.sum() == pytest.approx(-1.1520408898, rel=1e-9)


@pytest.mark.parametrize("sigma", [0.5, 0.8, 1.0, 1.4, 2.0, 5.0, 20.0, 100.0])
@pytest.mark.parametrize("q", [64, 512, 2048])
def test_mask_is_integer_zero_sum_d4(sigma, q):
    """Reading R1: integer, zero-sum, D4-symmetric masks scaled to max |w| ~ Q."""
    _, w = oracle.log_mask(sigma, q)
    assert np.all(w == np.round(w))
    assert w.sum() == 0
    for t in (w.T, w[::-1, :], w[:, ::-1], np.rot90(w)):
        assert np.array_equal(t, w)
    assert abs(np.abs(w).max() - q) <= 12
    # the sign pattern of Eq. 1 survives: the centre is the most negative tap
    assert w[2, 2] == w.min() < 0


def test_mask_worked_values_q512():
    """Reading R1 worked values at Q = 512 (computed independently of this
    oracle when the reading was written): sigma 0.5 centre -516, rings
    r^2 = 1, 2, 4, 5, 8 -> 75, 33, 6, 5, 5; sigma 20 -> -383, -255, 1, 128, 510."""
    _, w1 = oracle.log_mask(0.5, 512)
    _, w2 = oracle.log_mask(20.0, 512)
    ring = lambda w: [w[2, 2], w[2, 3], w[1, 3], w[2, 4], w[1, 4], w[0, 4]]
    assert ring(w1) == [-516, 75, 33, 6, 5, 5]
    assert ring(w2) == [-516, -383, -255, 1, 128, 510]
    assert list(w1.sum(axis=0)) == [26, 151, -354, 151, 26]
    assert list(w2.sum(axis=0)) == [1277, -637, -1280, -637, 1277]


@pytest.mark.parametrize("sigma", [0.5, 0.7, 1.3, 20.0, 3.3])
def test_mask_brute_force_reconstruction(sigma):
    """The independent Python construction gives the same integer mask."""
    _, w = oracle.log_mask(sigma, 512)
    b = brute.log_mask(sigma, 512)
    for (dx, dy), v in b.items():
        assert w[dy + 2, dx + 2] == v


# ------------------------------------------------------- whole pipeline

@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (5, 5), (13, 9), (40, 33)])
@pytest.mark.parametrize("value,dtype", [(0, np.uint8), (255, np.uint8), (37, np.uint8),
                                         (65535, np.uint16), (4095, np.uint16)])
def test_constant_image_has_no_features(shape, value, dtype):
    """Zero-sum masks give L = 0 on a constant image; no crossing, no feature."""
    img = np.full(shape, value, dtype=dtype)
    p = params(t_zc=(-1.0, -1.0), t_sd5=(-1.0, -1.0), t_sd3=(-1.0, -1.0), t_sdmax=(-1.0, -1.0))
    out, st = oracle.extract(img, p, stages=True)
    assert not out.any()
    assert not st["L1"].any() and not st["L2"].any()
    assert not st["Z1"].any() and not st["Z2"].any()


def test_linear_ramp_interior_is_flat():
    """Symmetric zero-sum masks annihilate affine functions (second moments
    vanish on a linear ramp), so L = 0 away from the borders."""
    H, W = 24, 31
    y, x = np.mgrid[0:H, 0:W]
    img = (1000 + 37 * x + 11 * y).astype(np.uint16)
    _, st = oracle.extract(img, params(), stages=True)
    for name in ("L1", "L2"):
        assert not st[name][2:-2, 2:-2].any()
        assert not st["Z" + name[1]][3:-3, 3:-3].any()


def _step(a, b, H=30, W=40, x0=20, dtype=np.uint16):
    img = np.full((H, W), a, dtype=dtype)
    img[:, x0:] = b
    return img


@pytest.mark.parametrize("a,b", [(100, 160), (160, 100), (0, 4095), (4095, 1000), (20, 21)])
def test_step_edge_closed_forms(a, b):
    """Vertical step a | b at columns 19 | 20.  With colsums (c2, c1, c0, c1, c2)
    of the mask: L(18) = c2 D, L(19) = (c1+c2) D, L(20) = -(c1+c2) D,
    L(21) = -c2 D, zero elsewhere (D = b - a).  The tie |L(19)| = |L(20)| goes
    to the negative pixel, i.e. the bright side (Sec. 3.2, reading R3);
    s5 = s3 = |D|/2 exactly (Eq. 2)."""
    img = _step(a, b)
    D = b - a
    p = params(t_zc=(0.0, 0.0), t_sd5=(0.0, 0.0), t_sd3=(0.0, 0.0), t_sdmax=(1e9, 1e9), hmf=())
    out, st = oracle.extract(img, p, stages=True)
    for f, sig in ((1, 0.5), (2, 20.0)):
        _, w = oracle.log_mask(sig)
        c = w.sum(axis=0)
        c1, c2 = c[1], c[0]
        L = st[f"L{f}"]
        expect = np.zeros(40)
        expect[18], expect[19], expect[20], expect[21] = c2 * D, (c1 + c2) * D, -(c1 + c2) * D, -c2 * D
        assert np.array_equal(L, np.broadcast_to(expect, L.shape))
        line = 20 if D > 0 else 19
        Z = st[f"Z{f}"]
        assert Z[:, line].all() and Z.sum() == Z.shape[0]
    assert np.array_equal(out.any(axis=0).nonzero()[0], [20 if D > 0 else 19])
    assert out[:, 20 if D > 0 else 19].all()


@pytest.mark.parametrize("D", [40, -40])
@pytest.mark.parametrize("transpose", [False, True])
def test_crossing_map_deviation_closed_forms(D, transpose):
    """Standard deviation over the zero-crossing map (reading R4, source 1) on a
    step edge.  The crossing map is one full line, so the 5x5 window of a line
    pixel holds n = 5 crossings and its 3x3 window n = 3 (borders replicate the
    line).  Eq. 2 over n ones and Lambda - n zeros gives
    D = Lambda sum z^2 - (sum z)^2 = n (Lambda - n): D5 = 5 x 20 = 100 and
    D3 = 3 x 6 = 18, so s5 = sqrt(100 / (25 x 24)) = sqrt(1/6) = 0.40825 and
    s3 = sqrt(18 / (9 x 8)) = 1/2."""
    img = _step(1000, 1000 + D)
    if transpose:
        img = np.ascontiguousarray(img.T)
    line = 20 if D > 0 else 19
    s5, s3 = math.sqrt(5 * 20 / (25 * 24)), math.sqrt(3 * 6 / (9 * 8))
    assert abs(s5 - math.sqrt(1 / 6)) < 1e-15 and s3 == 0.5

    def run(t5, tmax, t3):
        p = params(stddev_source=1, t_zc=(0.0, 0.0), t_sd5=(t5, t5), t_sdmax=(tmax, tmax), t_sd3=(t3, t3), hmf=())
        out = oracle.extract(img, p)
        return out.T if transpose else out

    full = np.zeros((30, 40), np.uint8)
    full[:, line] = 1
    # the 5x5 test decides while s5 <= t_sdmax
    assert np.array_equal(run(0.408, 10.0, 10.0), full)          # 0.408^2 x 600 = 99.9 < 100
    assert not run(0.409, 10.0, 0.0).any()                       # 0.409^2 x 600 = 100.4 > 100
    # above t_sdmax the 3x3 window decides: s3 = 1/2
    assert np.array_equal(run(10.0, 0.3, 0.49), full)            # 0.49^2 x 72 = 17.3 < 18
    assert not run(0.0, 0.3, 0.51).any()                         # 0.51^2 x 72 = 18.7 > 18
    assert not run(0.0, 0.3, 0.5).any()                          # s3 > 1/2 is strict
    # brute force agrees on the same image
    p = params(stddev_source=1, t_zc=(0.0, 0.0), t_sd5=(0.408, 0.408), t_sdmax=(10.0, 10.0),
               t_sd3=(10.0, 10.0), hmf=())
    assert np.array_equal(oracle.extract(img, p), _brute(img, p))


@pytest.mark.parametrize("hmf", [(), (5,), (3,)])
@pytest.mark.parametrize("a,b", [(100, 160), (160, 100)])
def test_tiny_images_hand_cases(a, b, hmf):
    """Hand-derived results for the smallest images (reading R2: every stage
    replicates its border).  A 1 x N row with a step, its N x 1 transpose and
    the 2 x 2 steps all extend to an unbounded straight step edge, so each
    gives the step-edge line of Sec. 3.2 at the bright-side pixel and nothing
    else (a one-pixel line survives the hybrid median: the '+' group holds the
    line's replicated column, 5 of 9); a 1 x 1 or constant image gives
    nothing."""
    p = params(t_zc=(0.0, 0.0), t_sd5=(0.0, 0.0), t_sd3=(0.0, 0.0), t_sdmax=(1e9, 1e9), hmf=hmf)
    bright = 1 if b > a else 0
    row = np.full((1, 40), a, np.uint16)
    row[:, 20:] = b
    out = oracle.extract(row, p)
    assert np.array_equal(out.nonzero()[1], [20 if b > a else 19])
    assert np.array_equal(oracle.extract(row.reshape(40, 1), p), out.T)
    sq = np.array([[a, b], [a, b]], np.uint16)
    expect = np.zeros((2, 2), np.uint8)
    expect[:, bright] = 1
    assert np.array_equal(oracle.extract(sq, p), expect)
    assert np.array_equal(oracle.extract(np.ascontiguousarray(sq.T), p), expect.T)
    for img in (np.array([[a]], np.uint16), np.full((2, 2), b, np.uint16), np.full((1, 7), a, np.uint16)):
        assert not oracle.extract(img, p).any()


@pytest.mark.parametrize("D", [13, 24, 100, -40])
def test_step_edge_threshold_boundaries(D):
    """Exactness of the strict thresholds on the step edge: contrast
    max - min of (c1+c2) D, -(c1+c2) D, -c2 D (that is 2 (c1+c2) |D| for
    sigma 0.5 but (c1 + 2 c2) |D| for sigma 20, where |c2| > |c1+c2|), and
    s = |D|/2 (Eq. 2 closed form for 10+15 and 3+6 pixels)."""
    img = _step(1000, 1000 + D)
    line = 20 if D > 0 else 19
    s = abs(D) / 2

    def contrast(sig):
        # L on the line pixel and its W / E neighbours from the closed forms
        # (N and S repeat the line value): max - min of those three values
        c = oracle.log_mask(sig)[1].sum(axis=0)
        L = {18: c[0] * D, 19: (c[1] + c[0]) * D, 20: -(c[1] + c[0]) * D, 21: -c[0] * D}
        v = [L.get(line - 1, 0), L[line], L.get(line + 1, 0)]
        return max(v) - min(v)

    c_1, c_2 = contrast(0.5), contrast(20.0)
    assert c_1 == 2 * 177 * abs(D) and c_2 == (640 + 1277) * abs(D)
    base = dict(t_sdmax=(1e9, 1e9), hmf=())
    # contrast exactly at threshold fails, one below passes (per branch)
    for tz, expect in (((c_1, c_2), False), ((c_1 - 1, 1e12), True), ((1e12, c_2 - 1), True)):
        out = oracle.extract(img, params(t_zc=tz, t_sd5=(0, 0), t_sd3=(0, 0), **base))
        assert bool(out[:, line].all()) == expect and out.sum() == (30 if expect else 0)
    # standard deviation exactly at threshold fails, just below passes
    for ts, expect in ((s, False), (math.nextafter(s, 0), True)):
        out = oracle.extract(img, params(t_zc=(0, 0), t_sd5=(ts, ts), t_sd3=(ts, ts), **base))
        assert bool(out[:, line].all()) == expect
    # above t_sdmax the 3x3 window decides (s3 = s5 here)
    out = oracle.extract(img, params(t_zc=(0, 0), t_sd5=(1e9, 1e9), t_sdmax=(0, 0),
                                     t_sd3=(s, s), hmf=()))
    assert not out.any()
    out = oracle.extract(img, params(t_zc=(0, 0), t_sd5=(1e9, 1e9), t_sdmax=(0, 0),
                                     t_sd3=(s - 0.5, s - 0.5), hmf=()))
    assert out[:, line].all()


def test_horizontal_step_is_transpose():
    img = _step(100, 190, H=40, W=30, x0=17).T.copy()
    out = oracle.extract(img, params(hmf=(5,)))
    assert np.array_equal(out.any(axis=1).nonzero()[0], [17])


def test_zero_response_crossing_rule():
    """Reading R3, exact zeros: an odd profile around column 10 gives L(10) = 0
    with L(9) and L(11) of opposite signs; the crossing sits on the zero."""
    prof = np.array([100] * 10 + [150] + [200] * 10, dtype=np.uint16)
    img = np.tile(prof, (12, 1))
    _, st = oracle.extract(img, params(t_zc=(0, 0), t_sd5=(0, 0), t_sd3=(0, 0), hmf=()), stages=True)
    for f in (1, 2):
        L = st[f"L{f}"]
        assert (L[:, 10] == 0).all() and (L[:, 9] * L[:, 11] < 0).all()
        assert np.array_equal(st[f"Z{f}"].any(axis=0).nonzero()[0], [10])


# ------------------------------------------------------ hybrid median

def _tile_patterns(patterns, k):
    """Pack k x k windows into one image, window i at tile i (tiles are k x k)."""
    n = len(patterns)
    cols = 256
    rows = (n + cols - 1) // cols
    img = np.zeros((rows * k, cols * k), dtype=patterns.dtype)
    for i in range(n):
        r, c = divmod(i, cols)
        img[r * k:(r + 1) * k, c * k:(c + 1) * k] = patterns[i]
    return img, cols


def _hmf_expect(win, k):
    r = k // 2
    plus = [win[r, r + d] for d in range(-r, r + 1)] + [win[r + d, r] for d in range(-r, r + 1) if d]
    cross = [win[r + d, r + d] for d in range(-r, r + 1)] + [win[r - d, r + d] for d in range(-r, r + 1) if d]
    return int(np.median([np.median(plus), np.median(cross), win[r, r]]))


@pytest.mark.parametrize("k", [3, 5])
def test_hmf_exhaustive_binary(k):
    """Sec. 3.4: every binary pattern on the '+' and 'x' subgroups (2^17 for
    k = 5, 2^9 for k = 3) against numpy's median of each subgroup and of the
    three values."""
    r = k // 2
    cells = [(r, r)] + [(r, r + d) for d in range(-r, r + 1) if d] + \
            [(r + d, r) for d in range(-r, r + 1) if d] + \
            [(r + d, r + d) for d in range(-r, r + 1) if d] + \
            [(r - d, r + d) for d in range(-r, r + 1) if d]
    n = 1 << len(cells)
    bits = ((np.arange(n)[:, None] >> np.arange(len(cells))[None, :]) & 1).astype(np.uint8)
    pats = np.zeros((n, k, k), dtype=np.uint8)
    for j, (y, x) in enumerate(cells):
        pats[:, y, x] = bits[:, j]
    img, cols = _tile_patterns(pats, k)
    out = oracle.hybrid_median(img, k)
    centres = out[r::k, r::k].reshape(-1)[:n]
    # vectorised medians: binary median of an odd count = majority
    plus_idx = [0] + list(range(1, 1 + 4 * r))
    cross_idx = [0] + list(range(1 + 4 * r, 1 + 8 * r))
    mp = (bits[:, plus_idx].sum(1) * 2 > len(plus_idx)).astype(int)
    mx = (bits[:, cross_idx].sum(1) * 2 > len(cross_idx)).astype(int)
    expect = ((mp + mx + bits[:, 0]) >= 2).astype(np.uint8)
    assert np.array_equal(centres, expect)
    # spot-check the majority shortcut itself against np.median on windows
    for i in np.random.default_rng(1).integers(0, n, 200):
        assert _hmf_expect(pats[i], k) == expect[i]


def test_hmf7_random_binary_patterns():
    """Window 7 (13 pixels in each subgroup, 25 distinct cells): 2^25 patterns
    are too many to enumerate, so 120000 random ones with a random density per
    pattern (every count of ones occurs), against the subgroup majorities, and
    a spot check of those against numpy's median on the windows."""
    k, r = 7, 3
    cells = [(r, r)] + [(r, r + d) for d in range(-r, r + 1) if d] + \
            [(r + d, r) for d in range(-r, r + 1) if d] + \
            [(r + d, r + d) for d in range(-r, r + 1) if d] + \
            [(r - d, r + d) for d in range(-r, r + 1) if d]
    assert len(cells) == 25
    rng = np.random.default_rng(77)
    n = 120000
    dens = rng.random(n)[:, None]
    bits = (rng.random((n, 25)) < dens).astype(np.uint8)
    pats = rng.integers(0, 2, size=(n, k, k)).astype(np.uint8)  # cells off the groups are noise
    for j, (y, x) in enumerate(cells):
        pats[:, y, x] = bits[:, j]
    img, cols = _tile_patterns(pats, k)
    out = oracle.hybrid_median(img, k)
    centres = out[r::k, r::k].reshape(-1)[:n]
    plus_idx = [0] + list(range(1, 13))
    cross_idx = [0] + list(range(13, 25))
    mp = (bits[:, plus_idx].sum(1) >= 7).astype(int)
    mx = (bits[:, cross_idx].sum(1) >= 7).astype(int)
    expect = ((mp + mx + bits[:, 0]) >= 2).astype(np.uint8)
    assert np.array_equal(centres, expect)
    assert len(set(bits[:, plus_idx].sum(1))) == 14  # counts 0 .. 13 all occur
    for i in rng.integers(0, n, 300):
        assert _hmf_expect(pats[i], k) == expect[i]


@pytest.mark.parametrize("k", [5, 7])
def test_hmf_grayscale_against_numpy_median(k):
    rng = np.random.default_rng(5 + k)
    pats = rng.integers(0, 65536, size=(3000, k, k)).astype(np.uint16)
    img, cols = _tile_patterns(pats, k)
    out = oracle.hybrid_median(img, k)
    got = out[k // 2::k, k // 2::k].reshape(-1)[:3000]
    assert all(int(got[i]) == _hmf_expect(pats[i], k) for i in range(3000))


@pytest.mark.parametrize("k", [3, 5, 7])
def test_hmf_salt_pepper_and_lines(k):
    """Sec. 3.4 / Sec. 2: isolated impulses are removed, thin lines (axis and
    45 degrees) survive: on a line the '+' group holds k of its 2k - 1
    pixels (the line's column) and the centre is set, so the median keeps
    it; next to the line both groups hold at most one set pixel."""
    z = np.zeros((17, 17), np.uint8)
    s = z.copy(); s[8, 8] = 1
    assert not oracle.hybrid_median(s, k).any()
    p = np.ones_like(z); p[8, 8] = 0
    assert oracle.hybrid_median(p, k).all()
    v = z.copy(); v[:, 6] = 1
    assert np.array_equal(oracle.hybrid_median(v, k), v)
    d = np.eye(17, dtype=np.uint8)
    assert np.array_equal(oracle.hybrid_median(d, k), d)
    # a 2 x 2 speck is removed by window 7 (each group holds at most 3 of 13)
    q = z.copy(); q[8:10, 8:10] = 1
    if k == 7:
        assert not oracle.hybrid_median(q, k).any()


# ---------------------------------------------------------------- Eq. 2

def test_stddev_decision_matches_statistics_stdev():
    """Eq. 2 is the unbiased sample standard deviation: the oracle's S plane
    agrees with statistics.stdev on the (clamped) 5x5 / 3x3 windows wherever
    the value is not within 1e-9 of a threshold."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 4096, size=(23, 19)).astype(np.uint16)
    img[5:9, 3:15] = 2000  # some flat windows too
    t5, tmax, t3 = 400.0, 1100.0, 700.0
    p = params(t_sd5=(t5, t5), t_sdmax=(tmax, tmax), t_sd3=(t3, t3), hmf=())
    _, st = oracle.extract(img, p, stages=True)
    H, W = img.shape
    checked = 0
    for y in range(H):
        for x in range(W):
            win = lambda r: [int(img[min(max(y + dy, 0), H - 1), min(max(x + dx, 0), W - 1)])
                             for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
            s5, s3 = statistics.stdev(win(2)), statistics.stdev(win(1))
            if min(abs(s5 - t5), abs(s5 - tmax), abs(s3 - t3)) < 1e-9:
                continue
            expect = (s3 > t3) if s5 > tmax else (s5 > t5)
            assert st["S1"][y, x] == expect and st["S2"][y, x] == expect
            checked += 1
    assert checked > 400


# ------------------------------------------------------------ invariants

def _crop_scene(seed, H=48, W=56, bits=8):
    big = scenes.scene(160, 160, seed=seed, n_rects=30, noise_sigma=4 * (1 << max(bits - 8, 0)),
                       impulse_frac=0.01, bits=bits)
    return big[40:40 + H, 50:50 + W].copy()


D4 = [
    (lambda a: a, lambda a: a),
    (lambda a: np.rot90(a, 1), lambda a: np.rot90(a, -1)),
    (lambda a: np.rot90(a, 2), lambda a: np.rot90(a, -2)),
    (lambda a: np.rot90(a, 3), lambda a: np.rot90(a, -3)),
    (lambda a: a[::-1], lambda a: a[::-1]),
    (lambda a: a[:, ::-1], lambda a: a[:, ::-1]),
    (lambda a: a.T, lambda a: a.T),
    (lambda a: np.rot90(a, 1).T, lambda a: np.rot90(a.T, -1)),
]


@pytest.mark.parametrize("hmf", [(), (5,), (3,), (5, 3), (7,), (7, 5, 3)])
@pytest.mark.parametrize("source", [0, 1])
def test_dihedral_equivariance(hmf, source):
    """The masks, the 4-neighbourhood, the windows and the '+'/'x' subgroups
    are all D4-invariant, and replicated borders commute with D4, so the
    pipeline is D4-equivariant."""
    img = _crop_scene(3)
    p = params(hmf=hmf, stddev_source=source)
    if source == 1:
        p.update(t_sd5=(0.3, 0.3), t_sdmax=(0.45, 0.45), t_sd3=(0.4, 0.4))
    ref = oracle.extract(img, p)
    assert ref.any()
    for fwd, inv in D4:
        out = oracle.extract(np.ascontiguousarray(fwd(img)), p)
        assert np.array_equal(inv(out), ref)


def test_offset_invariance():
    """Zero-sum masks and standard deviations ignore a constant offset."""
    img = _crop_scene(4, bits=12)
    p = params()
    p.update(oracle.default_params(16.0))
    ref = oracle.extract(img, p)
    assert ref.any()
    for c in (1, 17, 300):
        assert np.array_equal(oracle.extract((img.astype(np.int64) + c).astype(np.uint16), p), ref)


def test_gain_scaling():
    """L and s scale by an integer gain g; scaling the thresholds by g keeps the mask."""
    img = _crop_scene(6)
    p = oracle.default_params(1.0)
    ref = oracle.extract(img, p)
    for g in (2, 3, 16, 200):
        pg = oracle.default_params(float(g))
        assert np.array_equal(oracle.extract(img.astype(np.uint16) * np.uint16(g), pg), ref)


def test_interior_translation():
    """Away from the borders (radius 5: LoG 2 + crossing 1 + median 2), a crop
    sees the same mask as the full image."""
    big = scenes.scene(96, 80, seed=9, n_rects=20, noise_sigma=4, impulse_frac=0.01, bits=8)
    full = oracle.extract(big, params())
    for oy, ox in ((7, 11), (20, 3), (0, 0)):
        crop = big[oy:oy + 50, ox:ox + 60].copy()
        out = oracle.extract(crop, params())
        assert np.array_equal(out[5:-5, 5:-5], full[oy + 5:oy + 45, ox + 5:ox + 55])


def test_row_window_matches_full():
    img = _crop_scene(12, H=61, W=37)
    for hmf in ((), (5,), (5, 3)):
        p = params(hmf=hmf)
        full = oracle.extract(img, p)
        for y0, y1 in ((0, 1), (0, 9), (3, 17), (50, 61), (60, 61)):
            assert np.array_equal(oracle.extract(img, p, rows=(y0, y1)), full[y0:y1])


def test_pitched_input_matches_contiguous():
    img = _crop_scene(13, H=20, W=33, bits=12)
    view = scenes.pitched(img, 256, fill=4095)
    p = oracle.default_params(16.0)
    assert np.array_equal(oracle.extract(view, p), oracle.extract(img, p))


# ---------------------------------------------------------- brute force

def _brute(img, p):
    return np.array(brute.Brute(img.tolist(), p).output(), dtype=np.uint8)


def test_brute_force_all_3x3_images():
    """All 3^9 images of size 3x3 with values in {0, 100, 200}: oracle versus
    the independent per-pixel brute force (no median, low thresholds so that
    crossings and deviations actually fire)."""
    vals = np.array([0, 100, 200], dtype=np.uint8)
    p = params(t_zc=(20000.0, 60000.0), t_sd5=(30.0, 10.0), t_sdmax=(70.0, 60.0),
               t_sd3=(50.0, 20.0), hmf=())
    fired = 0
    for code in itertools.product(range(3), repeat=9):
        img = vals[np.array(code)].reshape(3, 3)
        got = oracle.extract(img, p)
        exp = _brute(img, p)
        assert np.array_equal(got, exp), img
        fired += int(got.any())
    assert fired > 1000


@pytest.mark.parametrize("seed", range(18))
def test_brute_force_random_tiny_images(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 18)), int(rng.integers(1, 14))
    bits = int(rng.choice([8, 12]))
    img = rng.integers(0, 1 << bits, size=(H, W)).astype(np.uint8 if bits == 8 else np.uint16)
    if seed % 3 == 0:  # piecewise-constant blocks give exact zeros and ties
        img = np.repeat(np.repeat(img[: (H + 2) // 3, : (W + 2) // 3], 3, 0), 3, 1)[:H, :W].copy()
    sc = 1 << max(bits - 8, 0)
    p = dict(sigma=(0.5, 20.0), mask_q=512,
             t_zc=tuple(float(rng.integers(0, 60000 * sc)) for _ in range(2)),
             t_sd5=tuple(float(rng.integers(0, 40 * sc)) for _ in range(2)),
             t_sdmax=tuple(float(rng.integers(20 * sc, 90 * sc)) for _ in range(2)),
             t_sd3=tuple(float(rng.integers(0, 50 * sc)) for _ in range(2)),
             stddev_source=int(seed % 4 == 1),
             hmf=[(), (5,), (3,), (5, 3), (7,), (7, 5, 3)][seed % 6])
    if p["stddev_source"]:
        p.update(t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5), t_sd3=(0.3, 0.4))
    assert np.array_equal(oracle.extract(img, p), _brute(img, p))


def test_brute_force_scene_crop_with_median():
    img = _crop_scene(21, H=22, W=26)
    for hmf in ((5,), (5, 3), (3,)):
        p = params(hmf=hmf)
        got = oracle.extract(img, p)
        assert np.array_equal(got, _brute(img, p))


def test_brute_force_other_sigmas():
    img = _crop_scene(22, H=14, W=17)
    p = params(sigma=(1.0, 2.5), t_zc=(800.0, 900.0))
    assert np.array_equal(oracle.extract(img, p), _brute(img, p))


# ---------------------------------------------------------------- golden

def _read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    kv = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split(None, 1)
        kv[k] = v.strip()
    return kv


def test_golden_step_edge_worked_example():
    g = _read_golden("step_edge_u8.txt")
    W, H, sc = int(g["width"]), int(g["height"]), int(g["step_column"])
    img = np.full((H, W), int(g["left"]), dtype=np.uint8)
    img[:, sc:] = int(g["right"])
    expect = np.zeros((H, W), np.uint8)
    expect[:, int(g["expect_column"])] = 1
    assert np.array_equal(oracle.extract(img, oracle.default_params(1.0)), expect)
    assert np.array_equal(_brute(img, oracle.default_params(1.0)), expect)


@pytest.mark.skipif(__import__("platform").machine() != "x86_64",
                    reason="digest written on x86_64; numpy's SIMD float32 exp may differ in the last bit elsewhere")
def test_golden_pan512_digest():
    """Regression pin written by tests/golden/make_golden.py (oracle only)."""
    import hashlib
    g = _read_golden("pan512_u8_digest.txt")
    mask = oracle.extract(scenes.pan_512_u8(), oracle.default_params(1.0))
    assert hashlib.sha256(mask.tobytes()).hexdigest() == g["sha256"]
    assert [int(c) for c in g["row_counts"].split()] == list(mask.sum(axis=1))
