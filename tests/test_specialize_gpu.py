"""fx_specialize: the streaming first pass compiled at run time with one
parameter set's LoG ring weights and contrast thresholds as constants.  Its
masks must equal the precompiled kernel's and the oracle's for every strip
class, load mode and standard-deviation variant it serves."""
import numpy as np
import pytest
import torch

from gen import scenes
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _not_checked_build(cuda_lib):
    """The checked build's kernels count range-check failures in their own
    translation units, so it never specialises (FX_ERR_UNSUPPORTED)."""
    from paper_1304_3992_gb300 import fx
    if fx.checked_violations() is not None:
        pytest.skip("checked build: no run-time specialisation")


def _extract(fx, img, p):
    out = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    fx.extract(img, p, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    ("default", dict()),
    ("median 3 (compact strips)", dict(hmf=(3,))),
    ("no median (compact strips)", dict(hmf=())),
    ("median 7, 5, 3 (wide strips)", dict(hmf=(7, 5, 3))),
    ("median 7, 7, 7 (extra-wide strips)", dict(hmf=(7, 7, 7))),
    ("branch thresholds differ", dict(t_sd5=(5.0, 7.0), t_sd3=(4.0, 6.0), t_sdmax=(20.0, 30.0))),
    ("crossing-map deviation", dict(stddev_source=1, t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5), t_sd3=(0.3, 0.4))),
    ("other masks", dict(sigma=(0.8, 3.0), t_zc=(900.0, 400.0))),
]


@pytest.mark.parametrize("w", [1100, 1101])  # rows 4-byte aligned / not (packed odd width)
@pytest.mark.parametrize("bits", [12, 8])
@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_specialized_matches_generic_and_oracle(cuda_lib, name, kw, bits, w):
    from paper_1304_3992_gb300 import fx
    h = 700
    img = scenes.scene(w, h, seed=bits * 31 + len(name), n_rects=300, noise_sigma=4.0 * (1 << (bits - 8)),
                       impulse_frac=0.01, bits=bits)
    scale = float(1 << (bits - 8))
    dtype = fx.FX_U8 if bits == 8 else fx.FX_U16
    d = oracle.default_params(scale)
    d.update(kw)
    p = fx.params_from_dict(d, dtype)
    x = torch.from_numpy(img).cuda()
    generic = _extract(fx, x, p)
    assert fx.specialize(p, dtype), "run-time compilation unavailable"
    special = _extract(fx, x, p)
    assert np.array_equal(special, generic), f"{name}: {int((special != generic).sum())} pixels differ"
    ref = oracle.extract(img, d)
    assert np.array_equal(special, ref), f"{name}: {int((special != ref).sum())} pixels differ from the oracle"
    assert special.sum() > 0


def test_specialized_fp32_log_mode(cuda_lib):
    """The FP32-LoG mode (non-integer masks): specialised and precompiled
    kernels give the same masks."""
    from paper_1304_3992_gb300 import fx
    img = scenes.scene(900, 600, seed=5, n_rects=250, noise_sigma=16.0, impulse_frac=0.01, bits=12)
    p = fx.make_params(fx.FX_U16, 12, log_mode=fx.FX_LOG_FP32)
    x = torch.from_numpy(img).cuda()
    generic = _extract(fx, x, p)
    assert fx.specialize(p, fx.FX_U16)
    assert np.array_equal(_extract(fx, x, p), generic)


def test_specialized_full_band_seams(cuda_lib):
    """Band 0 of the benchmark, specialised (the benchmark's configuration):
    40-row bands across the first three unit seams, the top and bottom rows
    and one random band, against the oracle; then the whole band against the
    precompiled kernel's mask through another parameter object with the same
    values (the cache is keyed by value)."""
    import fullsize
    from paper_1304_3992_gb300 import fx
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    uh = fullsize.unit_height(16384, 16384, sms)
    band = next(iter(scenes.ms_bands_u16_12bit()))
    d = oracle.default_params(16.0)
    p = fx.params_from_dict(d, fx.FX_U16)
    x = torch.from_numpy(band).cuda()
    assert fx.specialize(p, fx.FX_U16)
    got = _extract(fx, x, p)
    for y0, y1 in fullsize.seam_bands(band.shape[0], uh, seed=3):
        ref = oracle.extract(band, d, rows=(y0, y1))
        assert np.array_equal(got[y0:y1], ref), f"rows {y0}:{y1}"
    p2 = fx.params_from_dict(dict(d), fx.FX_U16)
    assert np.array_equal(_extract(fx, x, p2), got)


def test_specialize_rejects_bad_arguments(cuda_lib):
    from paper_1304_3992_gb300 import fx
    p = fx.make_params(fx.FX_U16, 12)
    with pytest.raises(RuntimeError):
        fx.specialize(p, 7)
    # lists beyond the streaming kernel's radii (the general kernel) are not specialised
    assert not fx.specialize(fx.make_params(fx.FX_U16, 12, hmf=(7, 7, 7, 7)), fx.FX_U16)


@pytest.mark.parametrize("hmf", [(5,), (3,), (7, 5, 3), (7, 7, 7)])
def test_specialized_batched_path(cuda_lib, hmf):
    """Plans created after fx_specialize put the compiled group kernels in
    their graphs: uneven uint8 / uint16 scenes, the first three with
    256-byte pitches (aligned loads), the others packed (odd widths read
    pixel by pixel), batched, against single calls of the precompiled kernels
    and, on sampled bands, the oracle."""
    from paper_1304_3992_gb300 import fx
    batch = scenes.uneven_batch(n=6, lo=200, hi=1300, seed=21, master_side=1400)
    d = oracle.default_params(16.0)
    d["hmf"] = hmf
    p = fx.params_from_dict(d, fx.FX_U16)
    imgs = []
    for i, (v, _) in enumerate(batch):
        h, w = v.shape
        pitch = (w * v.itemsize + 255) // 256 * 256 if i < 3 else w * v.itemsize
        buf = torch.zeros((h, pitch // v.itemsize), dtype=torch.uint8 if v.itemsize == 1 else torch.uint16,
                          device="cuda")
        buf[:, :w] = torch.from_numpy(np.ascontiguousarray(v)).cuda()
        imgs.append(buf[:, :w])
    singles = [_extract(fx, x, p) for x in imgs]  # before any specialisation of these parameters
    assert fx.specialize(p, fx.FX_U16) and fx.specialize(p, fx.FX_U8)
    outs = [torch.full(x.shape, 9, dtype=torch.uint8, device="cuda") for x in imgs]
    with fx.Plan(p, max_images=8) as plan:
        plan.extract_batch(list(zip(imgs, outs)))
        torch.cuda.synchronize()
        assert plan.device_status() == 0
    for i, (o, single) in enumerate(zip(outs, singles)):
        assert np.array_equal(o.cpu().numpy(), single), f"scene {i}"
    d8 = oracle.default_params(16.0)
    d8["hmf"] = hmf
    for i in (0, 1):
        view = np.ascontiguousarray(batch[i][0])
        ref = oracle.extract(view, d8, rows=(0, min(64, view.shape[0])))
        assert np.array_equal(singles[i][:ref.shape[0]], ref), f"oracle scene {i}"
