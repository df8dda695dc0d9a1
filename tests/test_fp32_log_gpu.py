"""GPU parity of the FP32-LoG mode (non-integer masks, FP32 responses).

Against the exact oracle the bar is the FP32 parity rule (tests/tolerance.py):
differences only within the dependency radius of a decision whose exact
margin is below 1e-5 of the local response range, at most 1e-6 of the pixels
compared (zero on every case below a million pixels).  Among themselves the
GPU paths (streaming kernel, persistent batched kernel, general tile kernel
behind the allocation-free entry point) evaluate the same FP32 operations, so
their masks must be byte-identical.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gen import scenes

import tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pair(scale=1.0, **kw):
    from paper_1304_3992_gb300 import fx
    d = oracle.default_params(scale)
    d.update(log_mode=1)
    d.update(kw)
    return d, fx.params_from_dict(d)


def run(fx, img, p):
    out = fx.extract(dev(img) if not torch.is_tensor(img) else img, p)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def general_path(fx, p, imgs):
    """The general tile kernel (the allocation-free entry point runs it for
    every parameter set)."""
    pairs = [(dev(i), torch.full(i.shape, 7, dtype=torch.uint8, device="cuda")) for i in imgs]
    arr = (fx.ImageDesc * len(pairs))()
    for k, (img, out) in enumerate(pairs):
        arr[k] = fx.desc_for(img, out)
    rc = fx.load().fx_extract_batch_noalloc(ctypes.byref(p), arr, len(pairs),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return [o.cpu().numpy() for _, o in pairs]


def test_fp32_pan512_within_tolerance(cuda_lib):
    img = scenes.pan_512_u8()
    d, p = pair(1.0)
    got = run(cuda_lib, img, p)
    assert got.sum() > 1000
    assert tolerance.compare_with_oracle(img, got, d) == 0


SHAPES = [(1, 1), (1, 77), (64, 1), (5, 5), (17, 53), (52, 52), (97, 211), (203, 157)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bits", [8, 12, 16])
def test_fp32_ragged_sizes(cuda_lib, shape, bits):
    h, w = shape
    img = scenes.scene(w, h, seed=h * 1000 + w + bits, n_rects=max(1, h * w // 400), noise_sigma=3.0,
                       impulse_frac=0.01, bits=bits)
    d, p = pair(float(1 << max(bits - 8, 0)))
    got = run(cuda_lib, img, p)
    assert tolerance.compare_with_oracle(img, got, d) == 0


@pytest.mark.parametrize("case", range(11))
def test_fp32_parameter_variants(cuda_lib, case):
    """Median off / 3 / 5 then 3 / 7 and the crossing-map source (narrow
    streaming strips), median 5 then 5, 7 then 5 then 3 and three levels with
    the crossing-map source (wide strips), 7 then 7 then 7 (general tile
    kernel), other sigmas and mask scales."""
    img = scenes.scene(180, 140, seed=50 + case, n_rects=40, noise_sigma=16.0, impulse_frac=0.005, bits=12)
    kw = [dict(hmf=()), dict(hmf=(3,)), dict(hmf=(5, 3)),
          dict(stddev_source=1, t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5), t_sd3=(0.3, 0.4)),
          dict(sigma=(1.0, 2.5), t_zc=(9000.0, 20000.0)), dict(mask_q=1000, t_zc=(130000.0, 500000.0)),
          dict(hmf=(5, 5)), dict(hmf=(5, 3, 3), stddev_source=1, t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5),
                                 t_sd3=(0.3, 0.4)),
          dict(hmf=(7,)), dict(hmf=(7, 5, 3)), dict(hmf=(7, 7, 7))][case]
    d, p = pair(16.0, **kw)
    got = run(cuda_lib, img, p)
    assert tolerance.compare_with_oracle(img, got, d) == 0


@pytest.mark.parametrize("orient", ["vertical", "horizontal", "diagonal"])
def test_fp32_step_edges_keep_exact_ties(cuda_lib, orient):
    """On a clean step the two pixels of the crossing pair have exactly opposite
    responses; the FP32 evaluation from d_c = R_c - n_c I(p) keeps that exact,
    so the tie goes to the negative pixel as in the oracle."""
    H, W = 48, 64
    y, x = np.mgrid[0:H, 0:W]
    edge = {"vertical": x >= 30, "horizontal": y >= 21, "diagonal": x + y >= 50}[orient]
    img = np.where(edge, 3000, 1200).astype(np.uint16)
    d, p = pair(16.0, t_zc=(0.0, 0.0), t_sd5=(0.0, 0.0), t_sd3=(0.0, 0.0))
    got = run(cuda_lib, img, p)
    exp = oracle.extract(img, d)
    assert exp.sum() > 0
    assert np.array_equal(got, exp)


def test_fp32_gpu_paths_identical(cuda_lib):
    """Streaming, batched and general kernels give the same bytes, including
    16-bit values above 4095 (the wide pass of the streaming path)."""
    fx = cuda_lib
    d, p = pair(16.0)
    imgs = [np.ascontiguousarray(v) for v, _ in scenes.uneven_batch(n=6, lo=60, hi=600, seed=11, master_side=700)]
    rng = np.random.default_rng(3)
    wide = scenes.scene(333, 270, seed=12, n_rects=60, noise_sigma=200.0, impulse_frac=0.01, bits=16)
    wide[100:140, 50:90] = rng.integers(40000, 65536, size=(40, 40))
    imgs.append(wide)
    singles = [run(fx, i, p) for i in imgs]
    for i, (g, s) in enumerate(zip(general_path(fx, p, imgs), singles)):
        assert np.array_equal(g, s), f"general vs streaming, image {i}"
    pairs = [(dev(i), torch.zeros(i.shape, dtype=torch.uint8, device="cuda")) for i in imgs]
    with fx.Plan(p, max_images=8) as plan:
        plan.extract_batch(pairs)
        torch.cuda.synchronize()
        for i, ((_, out), s) in enumerate(zip(pairs, singles)):
            assert np.array_equal(out.cpu().numpy(), s), f"batched vs streaming, image {i}"
    # the wide image against the oracle too, with thresholds for 16-bit values
    dw, pw = pair(256.0)
    got = run(fx, wide, pw)
    assert got.sum() > 0
    assert tolerance.compare_with_oracle(wide, got, dw) == 0


def _sample_rows(H, rows, k, seed):
    rng = np.random.default_rng(seed)
    starts = [0, H - rows] + sorted(int(s) for s in rng.integers(rows, H - 2 * rows, k))
    return [(s, s + rows) for s in starts]


def test_fp32_ms8192_sampled_rows(cuda_lib):
    img = scenes.ms_8192_u16_11bit()
    d, p = pair(8.0)
    got = run(cuda_lib, img, p)
    for y0, y1 in _sample_rows(img.shape[0], 8, 8, 4):
        assert tolerance.compare_with_oracle(img, got[y0:y1], d, rows=(y0, y1)) == 0


def test_fp32_band16384_unit_seams_all_bands(cuda_lib):
    """The four 16384^2 bands in the FP32-LoG mode: 40-row bands across the
    first three unit seams, the top and bottom rows and one random band, under
    the parity rule (zero differing pixels expected)."""
    import fullsize
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    uh = fullsize.unit_height(16384, 16384, sms)
    d, p = pair(16.0)
    for b, band in enumerate(scenes.ms_bands_u16_12bit()):
        got = run(cuda_lib, band, p)
        for y0, y1 in fullsize.seam_bands(band.shape[0], uh, seed=10 + b):
            assert tolerance.compare_with_oracle(band, got[y0:y1], d, rows=(y0, y1)) == 0, f"band {b} rows {y0}:{y1}"


def test_fp32_tiny_log_rule_literal(cuda_lib):
    """The FP32-LoG mode against the literal parity rule (differences only where
    the exact |LoG| is below 1e-5 of the local response range, at most 1e-6 of
    the pixels) and the zero-difference bar every FP32 test holds: the 512^2
    scene in full, sampled rows of the 8192^2 scene."""
    img = scenes.pan_512_u8()
    d, p = pair(1.0)
    assert tolerance.compare_tiny_log_rule(img, run(cuda_lib, img, p), d) == 0
    big = scenes.ms_8192_u16_11bit()
    d, p = pair(8.0)
    got = run(cuda_lib, big, p)
    for y0, y1 in _sample_rows(big.shape[0], 16, 4, 9):
        assert tolerance.compare_tiny_log_rule(big, got[y0:y1], d, rows=(y0, y1)) == 0
