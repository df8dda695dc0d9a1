"""Pins of the oracle's FP32-LoG mode (reading R9: non-integer masks from
Eq. 1) and of the parity rule that compares the library's FP32 responses
with it (tests/tolerance.py).

The FP32 masks are pinned to Eq. 1 itself (through the raw samples, which
test_oracle_pins pins to closed forms), to the integer masks of reading R1,
and to the independent rational construction of brute.py; the extraction in
this mode to constant / affine / step-edge closed forms and to the brute
force on tiny images.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from gen import scenes

import tolerance


def params(**kw):
    p = oracle.default_params(1.0)
    p.update(log_mode=1)
    p.update(kw)
    return p


def _grid(q):
    e = 0
    while 2 ** e < q:
        e += 1
    return 2.0 ** (e - 23), e


@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.0, 20.0])
@pytest.mark.parametrize("q", [1, 64, 512, 1000, 4096])
def test_fp32_mask_on_grid_zero_sum_d4(sigma, q):
    """Reading R9: every weight a multiple of g = 2^(e-23) with |w| < 2^(e+1)
    (24 significant bits, exact in FP32); zero-sum exactly; D4-symmetric."""
    w = oracle.log_mask_fp32(sigma, q)
    g, e = _grid(q)
    m = w / g
    assert np.array_equal(m, np.round(m))
    assert np.abs(w).max() < 2.0 ** (e + 1)
    assert np.all(w.astype(np.float32).astype(np.float64) == w)
    assert math.fsum(w.ravel()) == 0.0
    for t in (w.T, w[::-1, :], w[:, ::-1], np.rot90(w)):
        assert np.array_equal(t, w)


@pytest.mark.parametrize("sigma", [0.5, 1.4, 20.0])
def test_fp32_mask_is_scaled_eq1(sigma):
    """Each off-centre weight is the mean-removed Eq. 1 sample scaled to
    max |w| = Q, to within half a grid step; the centre differs from its
    scaled sample by at most the 24 roundings of the others."""
    q = 512
    raw, _ = oracle.log_mask(sigma, q)
    c = raw - raw.mean()
    target = q * c / np.abs(c).max()
    w = oracle.log_mask_fp32(sigma, q)
    g, _ = _grid(q)
    off = np.ones((5, 5), bool)
    off[2, 2] = False
    assert np.all(np.abs(w - target)[off] <= g / 2 + 1e-12)
    assert abs(w[2, 2] - target[2, 2]) <= 24 * g / 2 + 1e-12


@pytest.mark.parametrize("sigma", [0.5, 20.0])
def test_fp32_and_integer_masks_agree(sigma):
    """Reading R1 rounds the same scaled samples to integers: every off-centre
    integer weight is the FP32 weight rounded half away from zero."""
    _, wi = oracle.log_mask(sigma, 512)
    wf = oracle.log_mask_fp32(sigma, 512)
    r = np.where(wf >= 0, np.floor(wf + 0.5), -np.floor(-wf + 0.5))
    off = np.ones((5, 5), bool)
    off[2, 2] = False
    assert np.array_equal(r[off], wi[off])


@pytest.mark.parametrize("sigma", [0.5, 20.0, 3.0])
def test_fp32_mask_brute_reconstruction(sigma):
    w = oracle.log_mask_fp32(sigma, 512)
    b = brute.log_mask_fp32(sigma, 512)
    assert sum(b.values()) == 0
    for (dx, dy), v in b.items():
        assert w[dy + 2, dx + 2] == float(v)


@pytest.mark.parametrize("shape,value", [((1, 1), 7), ((5, 9), 4000), ((13, 4), 0)])
def test_fp32_constant_image(shape, value):
    img = np.full(shape, value, dtype=np.uint16)
    out, st = oracle.extract(img, params(t_zc=(-1.0, -1.0), t_sd5=(-1.0, -1.0)), stages=True)
    assert not st["L1"].any() and not st["L2"].any()
    assert not out.any()


def test_fp32_linear_ramp_interior_is_flat():
    """Symmetric zero-sum masks annihilate affine functions; the grid masks
    are both, so L = 0 exactly away from the borders."""
    H, W = 20, 27
    y, x = np.mgrid[0:H, 0:W]
    img = (900 + 23 * x + 7 * y).astype(np.uint16)
    _, st = oracle.extract(img, params(), stages=True)
    assert not st["L1"][2:-2, 2:-2].any() and not st["L2"][2:-2, 2:-2].any()


@pytest.mark.parametrize("a,b", [(100, 160), (4095, 1000), (20, 21)])
def test_fp32_step_edge_closed_forms(a, b):
    """Vertical step a | b at columns 19 | 20 with the FP32 masks' column sums
    (c2, c1, c0, c1, c2): L(18) = c2 D, L(19) = (c1+c2) D, L(20) = -(c1+c2) D,
    L(21) = -c2 D; the tie goes to the negative pixel (reading R3)."""
    img = np.full((24, 40), a, dtype=np.uint16)
    img[:, 20:] = b
    D = b - a
    p = params(t_zc=(0.0, 0.0), t_sd5=(0.0, 0.0), t_sd3=(0.0, 0.0), t_sdmax=(1e9, 1e9), hmf=())
    out, st = oracle.extract(img, p, stages=True)
    for f, sig in ((1, 0.5), (2, 20.0)):
        c = oracle.log_mask_fp32(sig).sum(axis=0)
        c1, c2 = c[1], c[0]
        expect = np.zeros(40)
        expect[18], expect[19], expect[20], expect[21] = c2 * D, (c1 + c2) * D, -(c1 + c2) * D, -c2 * D
        assert np.array_equal(st[f"L{f}"], np.broadcast_to(expect, st[f"L{f}"].shape))
    line = 20 if D > 0 else 19
    assert np.array_equal(out.any(axis=0).nonzero()[0], [line])


def _brute(img, p):
    return np.array(brute.Brute(img.tolist(), p).output(), dtype=np.uint8)


def test_fp32_brute_force_3x3_sample():
    """1000 of the 3^9 images of size 3x3 over {0, 100, 200}: the oracle in
    the FP32-LoG mode versus the rational brute force."""
    vals = np.array([0, 100, 200], dtype=np.uint8)
    p = params(t_zc=(20000.0, 60000.0), t_sd5=(30.0, 10.0), t_sdmax=(70.0, 60.0),
               t_sd3=(50.0, 20.0), hmf=())
    codes = list(itertools.product(range(3), repeat=9))
    rng = np.random.default_rng(5)
    fired = 0
    for i in rng.choice(len(codes), 1000, replace=False):
        img = vals[np.array(codes[i])].reshape(3, 3)
        got = oracle.extract(img, p)
        assert np.array_equal(got, _brute(img, p)), img
        fired += int(got.any())
    assert fired > 50


@pytest.mark.parametrize("seed", range(8))
def test_fp32_brute_force_random_tiny_images(seed):
    rng = np.random.default_rng(100 + seed)
    H, W = int(rng.integers(1, 16)), int(rng.integers(1, 13))
    bits = int(rng.choice([8, 12, 16]))
    img = rng.integers(0, 1 << bits, size=(H, W)).astype(np.uint8 if bits == 8 else np.uint16)
    if seed % 3 == 0:
        img = np.repeat(np.repeat(img[: (H + 2) // 3, : (W + 2) // 3], 3, 0), 3, 1)[:H, :W].copy()
    sc = 1 << max(bits - 8, 0)
    p = params(t_zc=tuple(float(rng.uniform(0, 60000 * sc)) for _ in range(2)),
               t_sd5=tuple(float(rng.integers(0, 40 * sc)) for _ in range(2)),
               t_sdmax=tuple(float(rng.integers(20 * sc, 90 * sc)) for _ in range(2)),
               t_sd3=tuple(float(rng.integers(0, 50 * sc)) for _ in range(2)),
               stddev_source=int(seed % 4 == 1), hmf=[(), (5,), (3,), (5, 3)][seed % 4])
    if p["stddev_source"]:
        p.update(t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5), t_sd3=(0.3, 0.4))
    assert np.array_equal(oracle.extract(img, p), _brute(img, p))


def test_modes_agree_away_from_margins():
    """The two modes compute the same LoG up to mask rounding (at most half a
    unit of 512 per tap): on the 512^2 scene their masks differ on few pixels."""
    img = scenes.pan_512_u8()
    a = oracle.extract(img, oracle.default_params(1.0))
    b = oracle.extract(img, params())
    assert (a != b).mean() < 0.01
    assert a.sum() > 1000 and b.sum() > 1000


# ------------------------------------------------------- the parity rule

def test_tolerance_accepts_identical_and_rejects_planted_flip():
    img = scenes.pan_512_u8()[:64, :96].copy()
    p = params()
    exp = oracle.extract(img, p)
    assert tolerance.compare_with_oracle(img, exp.copy(), p) == 0
    _, st = oracle.extract(img, p, stages=True)
    exc = tolerance.excused_pixels([st["L1"], st["L2"]], p["t_zc"], tolerance.dependency_radius(p))
    ys, xs = np.nonzero(~exc)
    bad = exp.copy()
    bad[ys[0], xs[0]] ^= 1
    with pytest.raises(AssertionError):
        tolerance.compare_with_oracle(img, bad, p)


def test_tolerance_excuses_only_near_fragile_sites():
    """A planted near-zero response makes its neighbourhood (radius r_dep)
    excusable and nothing else; the cap still limits the count."""
    L = np.full((20, 20), 100.0)
    L[:, 10:] = -100.0                   # an edge: margins |L|, |L+L'| = 100 and 0 at the tie
    L[5, 3] = 1e-7                       # fragile: |L| << 1e-5 x range
    f = tolerance.fragile_sites(L, t_zc=50.0)
    assert f[5, 3]
    assert f[:, 9].all() and f[:, 10].all()   # the exact tie on the edge is fragile too
    assert not f[15, 3]
    exc = tolerance.dilate(f, 2)
    assert exc[7, 5] and not exc[8, 5] and not exc[15, 3]
    got = np.zeros((20, 20), np.uint8)
    exp = got.copy()
    got[7, 5] = 1
    assert tolerance.check(got, exp, exc, cap=1.0) == 1
    with pytest.raises(AssertionError):
        tolerance.check(got, exp, exc, cap=1e-6)
    got[15, 3] = 1
    with pytest.raises(AssertionError):
        tolerance.check(got, exp, exc, cap=1.0)


def test_tiny_log_rule_excuses_only_tiny_responses():
    """The literal rule: a difference is excused only at a pixel whose exact
    |L| is below 1e-5 of the range of L over its 5x5 window, in either branch;
    the edge pixels of a step (|L| = 100 against a range of 200) are not."""
    L1 = np.full((20, 20), 100.0)
    L1[:, 10:] = -100.0
    L1[5, 3] = 1e-7
    L2 = np.full((20, 20), 7.0)
    L2[12, 12] = 0.0                   # an exact zero inside a flat patch: range 7, excused
    exc = tolerance.tiny_log_excused([L1, L2])
    assert exc[5, 3] and exc[12, 12]
    assert not exc[5, 9] and not exc[5, 10] and not exc[0, 0]
    assert int(exc.sum()) == 2
    exp = np.zeros((20, 20), np.uint8)
    got = exp.copy()
    got[5, 3] = 1
    assert tolerance.check(got, exp, exc, cap=1.0) == 1
    got[5, 9] = 1
    with pytest.raises(AssertionError):
        tolerance.check(got, exp, exc, cap=1.0)


def test_tiny_log_rule_on_the_oracle_itself():
    img = scenes.pan_512_u8()[:64, :96].copy()
    p = params()
    exp = oracle.extract(img, p)
    assert tolerance.compare_tiny_log_rule(img, exp.copy(), p) == 0
    bad = exp.copy()
    _, st = oracle.extract(img, p, stages=True)
    ys, xs = np.nonzero(~tolerance.tiny_log_excused([st["L1"], st["L2"]]))
    bad[ys[0], xs[0]] ^= 1
    with pytest.raises(AssertionError):
        tolerance.compare_tiny_log_rule(img, bad, p)
