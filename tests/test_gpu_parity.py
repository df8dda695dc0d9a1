"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer/byte work, so the bar is bit-exactness: every compared mask byte must
be equal.  Small and ragged cases are compared in full; the full-size scenes
(8192^2 uint16 and one 16384^2 band, in the same launch configuration the
benchmark times) are compared on sampled row bands that include both image
borders, which the oracle computes on their own (its row-window mode).
"""
import numpy as np
import pytest

import oracle
from gen import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_pitched(a, pitch_bytes):
    h, w = a.shape
    buf = torch.zeros((h, pitch_bytes // a.itemsize), dtype=torch.uint8 if a.itemsize == 1 else torch.uint16,
                      device="cuda")
    buf[:, :w] = dev(a)
    return buf[:, :w]


def pair(scale=1.0, dtype_code=None, **kw):
    """Same parameters for the oracle (dict) and the library (fx.Params)."""
    from paper_1304_3992_gb300 import fx
    d = oracle.default_params(scale)
    d.update(kw)
    return d, fx.params_from_dict(d, dtype_code or fx.FX_U16)


def run(cuda_lib, img, p, **kw):
    out = cuda_lib.extract(dev(img) if not torch.is_tensor(img) else img, p, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def assert_same(got, ref, what=""):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError(f"{what}: {len(bad)} of {ref.size} pixels differ, first at {bad[:5].tolist()}")


def test_pan512_u8_bitexact(cuda_lib):
    img = scenes.pan_512_u8()
    d, p = pair(1.0)
    ref = oracle.extract(img, d)
    got = run(cuda_lib, img, p)
    assert ref.sum() > 1000
    assert_same(got, ref, "512^2 uint8")


SHAPES = [(1, 1), (1, 37), (41, 1), (2, 2), (5, 3), (7, 33), (33, 31), (65, 97), (100, 129),
          (31, 1000), (3, 517), (259, 6), (130, 161)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bits", [8, 12, 16])
def test_ragged_sizes(cuda_lib, shape, bits):
    h, w = shape
    rng = np.random.default_rng(h * 1000 + w + bits)
    big = scenes.scene(max(w, 16) + 20, max(h, 16) + 20, seed=int(rng.integers(1 << 30)),
                       n_rects=max(2, w * h // 600), noise_sigma=4.0 * (1 << max(0, min(bits, 12) - 8)),
                       impulse_frac=0.01, bits=min(bits, 12))
    img = big[7:7 + h, 9:9 + w].copy()
    if bits == 16:
        img = (img.astype(np.uint32) * 16 + rng.integers(0, 16, img.shape)).astype(np.uint16)
    scale = float(1 << max(0, bits - 8))
    for hmf in ((5,), (), (3,)):
        d, p = pair(scale, hmf=hmf)
        assert_same(run(cuda_lib, img, p), oracle.extract(img, d), f"{shape} bits={bits} hmf={hmf}")


@pytest.mark.parametrize("hmf", [(5,), (3,)])
@pytest.mark.parametrize("w", [1, 2, 31, 32, 33, 51, 52, 53, 55, 56, 57, 63, 64, 65, 95, 103, 104, 105, 111, 112,
                               113, 127, 129, 191, 257])
def test_widths_mod_tile(cuda_lib, w, hmf):
    """Widths around multiples of the narrow (52-column, median 5) and compact
    (56-column, median 3) strips and of the warp's 64-column window."""
    img = scenes.scene(w + 10, 90, seed=w, n_rects=10, noise_sigma=24, impulse_frac=0.005, bits=12)[:, 5:5 + w].copy()
    d, p = pair(16.0, hmf=hmf)
    assert_same(run(cuda_lib, img, p), oracle.extract(img, d), f"width {w} hmf {hmf}")


@pytest.mark.parametrize("pitch_extra", [0, 2, 256, 1000])
def test_pitched_rows(cuda_lib, pitch_extra):
    img = scenes.scene(301, 77, seed=3, n_rects=8, noise_sigma=24, impulse_frac=0.005, bits=12)
    pitch = 301 * 2 + pitch_extra
    d, p = pair(16.0)
    got = run(cuda_lib, dev_pitched(img, pitch), p)
    assert_same(got, oracle.extract(img, d), f"pitch {pitch}")


@pytest.mark.parametrize("bits", [8, 12, 16])
def test_odd_width_pair_and_fallback_loads(cuda_lib, bits):
    """Odd widths: with exactly width * elem bytes per row every lane loads its
    two pixels one by one; with room for one more pixel per row the last
    column is loaded as the aligned pair (W - 1, W), W being padding.  The
    padding holds the largest value of the type, which must neither reach the
    mask nor send the strip to the integer pass.  Both layouts against the
    oracle, on images taller than one work unit."""
    from paper_1304_3992_gb300 import fx
    for (h, w) in [(901, 333), (257, 1001), (64, 53)]:
        img = scenes.scene(w, h, seed=h + w + bits, n_rects=max(1, h * w // 500),
                           noise_sigma=4.0 * (1 << (bits - 8)), impulse_frac=0.005, bits=bits)
        scale = float(1 << (bits - 8)) if bits <= 12 else 16.0
        d, p = pair(scale, fx.FX_U8 if bits == 8 else fx.FX_U16)
        ref = oracle.extract(img, d)
        assert_same(run(cuda_lib, img, p), ref, f"{h}x{w} contiguous")
        elem = img.itemsize
        for pitch in ((w + 1) * elem if ((w + 1) * elem) % (2 * elem) == 0 else (w + 2) * elem,
                      ((w * elem + 255) // 256) * 256):
            top = 255 if elem == 1 else 65535
            buf = torch.full((h, pitch // elem), top, dtype=torch.uint8 if elem == 1 else torch.uint16, device="cuda")
            buf[:, :w] = dev(img)
            assert_same(run(cuda_lib, buf[:, :w], p), ref, f"{h}x{w} pitch {pitch}")


@pytest.mark.parametrize("w", [330, 331, 332, 333])
def test_uint8_word_loads(cuda_lib, w):
    """uint8 rows are read as the aligned 4-byte word holding each lane's
    pair when the base and pitch are multiples of 4 and the pitch reaches the
    end of the word holding the last pair; otherwise pixel by pixel.  Widths
    of every residue mod 4 with tight pitch, the smallest pitch that allows the
    word loads, a 256-byte pitch, and a base two bytes past an aligned address
    (the padding holds 255, which must not reach the mask), on images taller
    than one work unit, against the oracle."""
    from paper_1304_3992_gb300 import fx
    h = 901
    img = scenes.scene(w, h, seed=w, n_rects=h * w // 500, noise_sigma=4.0, impulse_frac=0.005, bits=8)
    d, p = pair(1.0, dtype_code=fx.FX_U8)
    ref = oracle.extract(img, d)
    assert ref.sum() > 0
    assert_same(run(cuda_lib, img, p), ref, f"{w} packed")
    word = ((w + (w & 1) + 3) // 4) * 4
    for pitch, off in ((word, 0), (256 * ((w + 255) // 256), 0), (word + 4, 2)):
        buf = torch.full((h, pitch + off), 255, dtype=torch.uint8, device="cuda")
        view = buf[:, off:off + w]
        view.copy_(dev(img))
        assert_same(run(cuda_lib, view, p), ref, f"{w} pitch {pitch} offset {off}")


def test_pitched_output(cuda_lib):
    img = scenes.scene(150, 60, seed=4, n_rects=8, noise_sigma=4, impulse_frac=0.01, bits=8)
    d, p = pair(1.0)
    buf = torch.full((60, 256), 7, dtype=torch.uint8, device="cuda")
    out = buf[:, :150]
    cuda_lib.extract(dev(img), p, out=out)
    torch.cuda.synchronize()
    assert_same(out.cpu().numpy(), oracle.extract(img, d), "pitched output")
    assert (buf[:, 150:].cpu().numpy() == 7).all(), "wrote past the row"


@pytest.mark.parametrize("case", range(10))
def test_parameter_variants(cuda_lib, case):
    rng = np.random.default_rng(100 + case)
    bits = [8, 12][case % 2]
    img = scenes.scene(173, 141, seed=200 + case, n_rects=20, noise_sigma=4.0 * (1 << (bits - 8)),
                       impulse_frac=0.01, bits=bits)
    sc = float(1 << (bits - 8))
    kw = dict(
        t_zc=(float(rng.integers(0, 9000)) * sc, float(rng.integers(0, 30000)) * sc),
        t_sd5=(float(rng.integers(0, 12)) * sc + 0.5, float(rng.integers(0, 12)) * sc),
        t_sdmax=(float(rng.integers(10, 40)) * sc, float(rng.integers(10, 40)) * sc),
        t_sd3=(float(rng.integers(0, 12)) * sc, float(rng.integers(0, 12)) * sc + 0.25),
        hmf=[(5,), (3,), (5, 3), (), (5, 5, 3), (3, 3)][case % 6],
        stddev_source=int(case in (3, 7)),
        sigma=[(0.5, 20.0), (0.7, 2.0), (1.0, 5.0)][case % 3],
    )
    if kw["stddev_source"]:
        kw.update(t_sd5=(0.3, 0.3), t_sdmax=(0.45, 0.45), t_sd3=(0.4, 0.4))
    d, p = pair(sc, **kw)
    assert_same(run(cuda_lib, img, p), oracle.extract(img, d), f"case {case}")


def test_negative_and_extreme_thresholds(cuda_lib):
    img = scenes.scene(120, 90, seed=8, n_rects=10, noise_sigma=24, impulse_frac=0.005, bits=12)
    for kw in (dict(t_zc=(-5.0, -1.0), t_sd5=(-1.0, -1.0), t_sdmax=(-1.0, -1.0), t_sd3=(-1.0, -1.0)),
               dict(t_zc=(1e30, 1e30)), dict(t_sd5=(1e300, 1e300), t_sdmax=(float("inf"),) * 2),
               dict(t_zc=(0.0, 0.0), t_sd5=(0.0, 0.0), t_sdmax=(0.0, 0.0), t_sd3=(0.0, 0.0))):
        d, p = pair(16.0, **kw)
        assert_same(run(cuda_lib, img, p), oracle.extract(img, d), str(kw))


def test_constant_and_step_images(cuda_lib):
    d, p = pair(16.0, t_zc=(0, 0), t_sd5=(0, 0), t_sd3=(0, 0))
    for h, w in ((1, 1), (37, 70)):
        assert not run(cuda_lib, np.full((h, w), 4095, np.uint16), p).any()
    step = np.full((40, 100), 1000, np.uint16)
    step[:, 61:] = 1200
    got = run(cuda_lib, step, p)
    assert np.array_equal(got.any(axis=0).nonzero()[0], [61]) and got[:, 61].all()


def test_dihedral_equivariance_gpu(cuda_lib):
    img = scenes.scene(211, 150, seed=12, n_rects=25, noise_sigma=24, impulse_frac=0.005, bits=12)
    _, p = pair(16.0)
    ref = run(cuda_lib, img, p)
    for fwd, inv in ((lambda a: a.T, lambda a: a.T), (lambda a: a[::-1], lambda a: a[::-1]),
                     (lambda a: np.rot90(a), lambda a: np.rot90(a, -1))):
        assert_same(inv(run(cuda_lib, np.ascontiguousarray(fwd(img)), p)), ref, "D4")


def _sample_bands(H, k, rows, seed):
    rng = np.random.default_rng(seed)
    starts = [0, H - rows] + sorted(int(s) for s in rng.integers(rows, H - 2 * rows, k))
    return [(s, s + rows) for s in starts]


def test_ms8192_u16_sampled_rows(cuda_lib):
    img = scenes.ms_8192_u16_11bit()
    d, p = pair(8.0)
    from paper_1304_3992_gb300 import fx
    p = fx.params_from_dict(d)
    got = run(cuda_lib, img, p)
    assert set(np.unique(got)) <= {0, 1}
    for y0, y1 in _sample_bands(img.shape[0], 6, 12, 1):
        assert_same(got[y0:y1], oracle.extract(img, d, rows=(y0, y1)), f"rows {y0}:{y1}")
    # left and right image borders over a tall band
    assert_same(got[3000:3100, :], oracle.extract(img, d, rows=(3000, 3100)), "rows 3000:3100")


def test_band16384_u16_unit_seams_all_bands(cuda_lib):
    """The benchmark's four 16384^2 12-bit bands, each in the benchmark's
    launch configuration: 40-row bands across the first three unit seams (656
    rows apart on 152 SMs), the top and bottom rows and one random band,
    against the oracle."""
    import fullsize
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    uh = fullsize.unit_height(16384, 16384, sms)
    if sms == 152:
        assert uh == 656
    d, p = pair(16.0)
    for b, band in enumerate(scenes.ms_bands_u16_12bit()):
        got = run(cuda_lib, band, p)
        for y0, y1 in fullsize.seam_bands(band.shape[0], uh, seed=b):
            assert_same(got[y0:y1], oracle.extract(band, d, rows=(y0, y1)), f"band {b} rows {y0}:{y1}")


@pytest.mark.parametrize("hmf", [(3,), ()])
def test_band16384_u16_compact_strips_seams(cuda_lib, hmf):
    """Band 0 of the benchmark with a window-3 median or none, which run on the
    compact strips (56 output columns): 40-row bands across the first three
    unit seams of that launch, the top and bottom rows and one random band,
    and the left and right image borders over a tall band, against the
    oracle."""
    import fullsize
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    uh = fullsize.unit_height(16384, 16384, sms, r_m=1)
    d, p = pair(16.0, hmf=hmf)
    band = next(iter(scenes.ms_bands_u16_12bit()))
    got = run(cuda_lib, band, p)
    for y0, y1 in fullsize.seam_bands(band.shape[0], uh, seed=5):
        assert_same(got[y0:y1], oracle.extract(band, d, rows=(y0, y1)), f"hmf {hmf} rows {y0}:{y1}")


def test_config4_batch_full_size_sampled(cuda_lib):
    """The 64 uneven scenes of the batched workload at full size (sides 1000 to
    12000, uint8 and 12-bit uint16, pitch rounded to 256 B) in one batched call;
    sampled row bands of four uint16 scenes (12-bit thresholds) and, from a
    second call with 8-bit thresholds, of four uint8 scenes against the
    oracle, and every scene's mask against its single-image call on a band."""
    batch = scenes.uneven_batch(n=64)
    imgs = [dev_pitched(view, view.strides[0]) for view, _ in batch]
    outs = [torch.full(view.shape, 9, dtype=torch.uint8, device="cuda") for view, _ in batch]
    rng = np.random.default_rng(64)
    for scale, dt, picks in ((16.0, np.uint16, (1, 3, 21, 63)), (1.0, np.uint8, (0, 2, 30, 62))):
        d, p = pair(scale)
        with cuda_lib.Plan(p, max_images=64) as plan:
            plan.extract_batch(list(zip(imgs, outs)))
            torch.cuda.synchronize()
            assert plan.device_status() == 0
        feats = 0
        for i in picks:
            view = batch[i][0]
            assert view.dtype == dt
            H = view.shape[0]
            y = int(rng.integers(16, H - 40))
            got = outs[i].cpu().numpy()
            for y0, y1 in ((0, 16), (y, y + 24), (H - 16, H)):
                ref = oracle.extract(view, d, rows=(y0, y1))
                assert_same(got[y0:y1], ref, f"scene {i} rows {y0}:{y1}")
                feats += int(ref.sum())
        assert feats > 0
        for i in range(0, 64, 7):  # batched output equals the single-image call
            single = cuda_lib.extract(imgs[i], p)
            torch.cuda.synchronize()
            assert torch.equal(single, outs[i]), f"scene {i}"


def test_batch_two_streams_one_plan(cuda_lib):
    """Two calls on one plan from two streams run without waiting for each
    other (the plan alternates between two descriptor tables and two sets of
    queue counters); both give the single-image masks."""
    batch = scenes.uneven_batch(n=12, lo=200, hi=1500, seed=12, master_side=1600)
    d, p = pair(16.0)
    pairs = [(dev_pitched(v, v.strides[0]), torch.full(v.shape, 9, dtype=torch.uint8, device="cuda"))
             for v, _ in batch]
    singles = [run(cuda_lib, img, p) for img, _ in pairs]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with cuda_lib.Plan(p, max_images=8) as plan:
        for rep in range(3):
            for _, o in pairs:
                o.fill_(9)
            torch.cuda.synchronize()
            plan.extract_batch(pairs[:6], stream=s1)
            plan.extract_batch(pairs[6:], stream=s2)
            torch.cuda.synchronize()
            for i, ((_, out), single) in enumerate(zip(pairs, singles)):
                assert_same(out.cpu().numpy(), single, f"rep {rep} image {i}")
        assert plan.device_status() == 0


def test_batch_matches_single_and_oracle(cuda_lib):
    batch = scenes.uneven_batch(n=10, lo=40, hi=700, seed=7, master_side=900)
    d, p = pair(16.0)
    d8 = oracle.default_params(16.0)
    pairs, singles = [], []
    for view, _ in batch:
        img = dev(view) if view.flags.c_contiguous else dev_pitched(view, view.strides[0])
        out = torch.full(view.shape, 9, dtype=torch.uint8, device="cuda")
        pairs.append((img, out))
        singles.append(run(cuda_lib, img, p))
    with cuda_lib.Plan(p, max_images=16) as plan:
        for rep in range(2):
            plan.extract_batch(pairs)
            torch.cuda.synchronize()
            for i, ((img, out), single) in enumerate(zip(pairs, singles)):
                assert_same(out.cpu().numpy(), single, f"batch image {i} rep {rep}")
        assert plan.device_status() == 0
    for i in (0, 1, 5):
        assert_same(singles[i], oracle.extract(np.ascontiguousarray(batch[i][0]), d8), f"oracle image {i}")


@pytest.mark.parametrize("hmf,uw", [((5,), 52), ((3,), 56), ((7, 5, 3), 44), ((5, 5), 44), ((), 56),
                                    ((7, 7, 7), 36)])
def test_batch_full_range_16bit_all_groups(cuda_lib, hmf, uw):
    """All four queue groups (uint16 / uint8, aligned pairs / pixel by pixel)
    in one batch, the uint16 images spanning the full 16-bit range: their
    strips are recomputed by the batched integer redo kernel (one resident
    wave striding over the units).  Each median list on its strip class
    (narrow 52, compact 56, wide 44 columns), with fixed unit shapes too.
    Against single-image calls and the oracle."""
    rng = np.random.default_rng(41)
    shapes = [(300, 420, 16), (257, 333, 16), (140, 1000, 8), (211, 97, 8), (90, 64, 16), (77, 53, 8)]
    imgs = []
    for h, w, bits in shapes:
        base = scenes.scene(w, h, seed=h + w, n_rects=max(1, h * w // 400), noise_sigma=4.0 * (1 << (bits - 8)),
                            impulse_frac=0.01, bits=bits)
        if bits == 16:  # push part of the image towards the top of the range
            base[: h // 2] = np.minimum(base[: h // 2].astype(np.int64) + 40000, 65535).astype(np.uint16)
        imgs.append(base)
    d, p = pair(4.0, hmf=hmf)  # features on every image: about 4 % of the uint8 pixels, 30 % of the uint16 ones
    pairs = [(dev(i), torch.full(i.shape, 9, dtype=torch.uint8, device="cuda")) for i in imgs]
    singles = [run(cuda_lib, img, p) for img, _ in pairs]
    with cuda_lib.Plan(p, max_images=8) as plan:
        with pytest.raises(RuntimeError):
            plan.set_tile(uw + 4, 0, 3)  # another class's width
        for shape in [None, (uw, 0, 3), (uw, 64, 1)]:
            if shape:
                plan.set_tile(*shape)
            for o in pairs:
                o[1].fill_(9)
            plan.extract_batch(pairs)
            torch.cuda.synchronize()
            for i, ((_, out), single) in enumerate(zip(pairs, singles)):
                assert_same(out.cpu().numpy(), single, f"batch image {i} tile {shape}")
        assert plan.device_status() == 0
    for i in (0, 1, 2):
        assert_same(singles[i], oracle.extract(imgs[i], d), f"oracle image {i}")


def test_batch_autotune_keeps_results(cuda_lib):
    batch = scenes.uneven_batch(n=6, lo=100, hi=900, seed=8, master_side=1000)
    _, p = pair(16.0)
    pairs = [(dev_pitched(v, v.strides[0]), torch.zeros(v.shape, dtype=torch.uint8, device="cuda")) for v, _ in batch]
    singles = [run(cuda_lib, img, p) for img, _ in pairs]
    with cuda_lib.Plan(p, max_images=8) as plan:
        cfg = plan.autotune(pairs)
        assert cfg[2] in (12, 10, 8)  # the streaming group kernels' candidates
        for o in pairs:
            o[1].zero_()
        plan.extract_batch(pairs)
        torch.cuda.synchronize()
        for (img, out), single in zip(pairs, singles):
            assert_same(out.cpu().numpy(), single, f"after autotune {cfg}")


def test_batch_set_tile_shapes_keep_results(cuda_lib):
    """Fixed unit heights (one that splits every image, one taller than all)
    and the automatic height (tile_h 0) give the same masks."""
    batch = scenes.uneven_batch(n=5, lo=80, hi=700, seed=9, master_side=800)
    _, p = pair(16.0)
    pairs = [(dev_pitched(v, v.strides[0]), torch.zeros(v.shape, dtype=torch.uint8, device="cuda")) for v, _ in batch]
    singles = [run(cuda_lib, img, p) for img, _ in pairs]
    with cuda_lib.Plan(p, max_images=8) as plan:
        # one-warp CTAs: 1 .. 32 per SM; 24 exceeds the resident count (the
        # CTAs beyond it start when earlier ones exit and find the queue empty)
        for shape in [(52, 16, 1), (52, 1024, 2), (52, 0, 3), (52, 0, 1), (52, 0, 12), (52, 512, 24)]:
            plan.set_tile(*shape)
            for o in pairs:
                o[1].fill_(9)
            plan.extract_batch(pairs)
            torch.cuda.synchronize()
            for (img, out), single in zip(pairs, singles):
                assert_same(out.cpu().numpy(), single, f"tile {shape}")
        assert plan.device_status() == 0


def test_extract_host_matches_device(cuda_lib):
    img = scenes.scene(1500, 1300, seed=31, n_rects=200, noise_sigma=24, impulse_frac=0.005, bits=12)
    _, p = pair(16.0)
    ref = run(cuda_lib, img, p)
    with cuda_lib.Plan(p, max_images=1) as plan:
        got = plan.extract_host(img)
        assert_same(got, ref, "host path")
        img8 = scenes.scene(999, 700, seed=32, n_rects=90, noise_sigma=4, impulse_frac=0.01, bits=8)
        assert_same(plan.extract_host(img8), run(cuda_lib, img8, p), "host path u8")


def test_device_pointer_checks(cuda_lib):
    import ctypes
    from paper_1304_3992_gb300 import fx
    lib = fx.load()
    p = fx.make_params(fx.FX_U16)
    host = np.zeros((8, 8), np.uint16)
    out = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    assert lib.fx_extract(host.ctypes.data, 8, 8, 16, fx.FX_U16, ctypes.byref(p), out.data_ptr(), None) == 1
    q = fx.make_params(fx.FX_U16, mask_q=1 << 20)
    img = torch.zeros((8, 8), dtype=torch.uint16, device="cuda")
    assert lib.fx_extract(img.data_ptr(), 8, 8, 16, fx.FX_U16, ctypes.byref(q), out.data_ptr(), None) == 3
    nanp = fx.make_params(fx.FX_U16, t_zc=(float("nan"), 0.0))
    assert lib.fx_extract(img.data_ptr(), 8, 8, 16, fx.FX_U16, ctypes.byref(nanp), out.data_ptr(), None) == 1


@pytest.mark.parametrize("hmf", [(5, 3), (3, 5), (3, 3), (7,), (3, 3, 3), (5, 5), (7, 5, 3), (7, 7),
                                 (5, 3, 3, 3), (3, 3, 3, 3), (7, 7, 7), (7, 7, 5, 3), (7, 7, 7, 7)])
def test_median_lists_streaming(cuda_lib, hmf):
    """Median lists (Sec. 3.4 windows 3, 5, 7; Sec. 4.2's repeated passes):
    radii adding up to 1 run on the compact streaming strips, 2 and 3 on the
    narrow ones, 4 to 7 on the wide ones, 8 to 11 on the extra-wide ones
    (7, 7, 7 and 7, 7, 5, 3) and 7, 7, 7, 7 (radius 12) on the general tile
    kernel; full masks of images taller than one work unit, both dtypes,
    against the oracle, and the batched plan against single calls."""
    imgs = [scenes.scene(700, 1100, seed=61, n_rects=300, noise_sigma=24.0, impulse_frac=0.01, bits=12),
            scenes.scene(1030, 613, seed=62, n_rects=250, noise_sigma=4.0, impulse_frac=0.01, bits=8)]
    d, p = pair(16.0, hmf=hmf)
    singles = []
    for img in imgs:
        dd = dict(d) if img.dtype == np.uint16 else dict(oracle.default_params(1.0), hmf=hmf)
        pp = p if img.dtype == np.uint16 else cuda_lib.params_from_dict(dd)
        got = run(cuda_lib, img, pp)
        assert_same(got, oracle.extract(img, dd), f"hmf {hmf} {img.dtype}")
        singles.append((img, pp, got))
    img, pp, ref = singles[0]
    pairs = [(dev(img), torch.zeros(img.shape, dtype=torch.uint8, device="cuda"))]
    with cuda_lib.Plan(pp, max_images=2) as plan:
        plan.extract_batch(pairs)
        torch.cuda.synchronize()
        assert_same(pairs[0][1].cpu().numpy(), ref, f"batched hmf {hmf}")


@pytest.mark.parametrize("hmf", [(5,), (5, 3), (3,), (), (7,), (5, 5), (7, 5, 3)])
def test_crossing_map_source_streaming(cuda_lib, hmf):
    """Standard deviation over the crossing map (reading R4, source 1) on the
    streaming kernel (48-column strips, bit-sliced window counts): full masks of
    images taller than one work unit, both dtypes, against the oracle, and the
    batched plan against single calls."""
    kw = dict(stddev_source=1, t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5), t_sd3=(0.3, 0.4), hmf=hmf)
    imgs = [scenes.scene(701, 1090, seed=71, n_rects=300, noise_sigma=24.0, impulse_frac=0.01, bits=12),
            scenes.scene(1030, 613, seed=72, n_rects=250, noise_sigma=4.0, impulse_frac=0.01, bits=8)]
    outs = []
    for img in imgs:
        scale = 16.0 if img.dtype == np.uint16 else 1.0
        d, p = pair(scale, **kw)
        got = run(cuda_lib, img, p)
        assert got.sum() > 0
        assert_same(got, oracle.extract(img, d), f"hmf {hmf} {img.dtype}")
        outs.append((img, p, got))
    img, p, ref = outs[0]
    pairs = [(dev(img), torch.zeros(img.shape, dtype=torch.uint8, device="cuda"))]
    with cuda_lib.Plan(p, max_images=2) as plan:
        plan.extract_batch(pairs)
        torch.cuda.synchronize()
        assert_same(pairs[0][1].cpu().numpy(), ref, f"batched hmf {hmf}")


def test_extract_host_batch_matches_device(cuda_lib):
    """fx_extract_host_batch: several host images (contiguous rows -> linear
    copies, padded rows -> pitched copies, both dtypes, one image of several
    chunks) through one pipeline, each equal to the device path."""
    imgs = [scenes.scene(1500, 1300, seed=41, n_rects=200, noise_sigma=24, impulse_frac=0.005, bits=12),
            scenes.scene(999, 700, seed=42, n_rects=90, noise_sigma=4, impulse_frac=0.01, bits=8),
            scenes.scene(4096, 9000, seed=43, n_rects=900, noise_sigma=24, impulse_frac=0.005, bits=12)]
    padded = scenes.pitched(imgs[1], 1280)
    hosts = [imgs[0], padded, imgs[2]]
    _, p = pair(16.0)
    outs = [np.full(h.shape, 9, np.uint8) for h in hosts]
    with cuda_lib.Plan(p, max_images=4) as plan:
        plan.extract_host_batch(list(zip(hosts, outs)))
        for i, (h, o) in enumerate(zip(hosts, outs)):
            assert_same(o, run(cuda_lib, np.ascontiguousarray(h), p), f"host batch image {i}")
        # a second call reuses the staging buffers
        outs2 = [np.zeros_like(o) for o in outs]
        plan.extract_host_batch(list(zip(hosts, outs2)))
        for o, o2 in zip(outs, outs2):
            assert_same(o2, o, "second call")


def test_extract_host_chunk_schedule(cuda_lib):
    """One 8192^2 uint16 image through the host path: a quarter-size first
    chunk, full chunks, a shortened chunk and a quarter-size last chunk (from
    page-locked and from pageable buffers), equal to the device path."""
    img = scenes.ms_8192_u16_11bit()
    d, p = pair(8.0)
    ref = run(cuda_lib, img, p)
    pinned_in = torch.from_numpy(img).pin_memory()
    pinned_out = torch.full(img.shape, 9, dtype=torch.uint8).pin_memory()
    pageable_out = np.full(img.shape, 9, np.uint8)
    with cuda_lib.Plan(p, max_images=2) as plan:
        plan.extract_host_batch([(pinned_in.numpy(), pinned_out.numpy())])
        assert_same(pinned_out.numpy(), ref, "pinned")
        plan.extract_host_batch([(img, pageable_out)])
        assert_same(pageable_out, ref, "pageable")


@pytest.mark.parametrize("hmf", [(), (5,), (3,), (7,), (7, 5, 3)])
def test_tiny_images_hand_cases_gpu(cuda_lib, hmf):
    """The hand-derived tiny cases of the oracle pins through the library: a
    one-row step, its one-column transpose and the 2 x 2 steps give the
    step-edge line at the bright-side pixel; constant tiny images give nothing."""
    d, p = pair(1.0, t_zc=(0.0, 0.0), t_sd5=(0.0, 0.0), t_sd3=(0.0, 0.0), t_sdmax=(1e9, 1e9), hmf=hmf)
    for a, b in ((100, 160), (160, 100)):
        row = np.full((1, 40), a, np.uint16)
        row[:, 20:] = b
        sq = np.array([[a, b], [a, b]], np.uint16)
        for img in (row, row.reshape(40, 1), sq, np.ascontiguousarray(sq.T), np.full((1, 1), a, np.uint16)):
            got = run(cuda_lib, img, p)
            assert_same(got, oracle.extract(img, d), f"{img.shape} {a}|{b} hmf={hmf}")
        assert run(cuda_lib, row, p).nonzero()[1].tolist() == [20 if b > a else 19]


@pytest.mark.parametrize("hmf", [(7,), (5, 5), (7, 5, 3), (7, 7, 7), (7, 7, 7, 5)])
@pytest.mark.parametrize("shape", [(1, 1), (2, 45), (45, 2), (31, 44), (97, 89), (203, 157), (77, 133), (50, 37)])
def test_ragged_sizes_window7_and_wide(cuda_lib, shape, hmf):
    """Window 7 and wide median lists on ragged sizes (widths around the 44-,
    36- and 52-column strips, single rows and columns) against the oracle;
    7, 7, 7 and 7, 7, 7, 5 (radii 9 and 11) run on the extra-wide strips."""
    h, w = shape
    img = scenes.scene(w, h, seed=h * 7 + w, n_rects=max(1, h * w // 300), noise_sigma=24.0,
                       impulse_frac=0.01, bits=12)
    d, p = pair(16.0, hmf=hmf)
    assert_same(run(cuda_lib, img, p), oracle.extract(img, d), f"{shape} hmf {hmf}")


def test_wide_strips_full_range_16bit(cuda_lib):
    """Values above the FP32-exact bound on the wide strips: the integer pass
    recomputes the marked strips (median 7, 5, 3)."""
    rng = np.random.default_rng(17)
    img = scenes.scene(333, 801, seed=23, n_rects=400, noise_sigma=64.0, impulse_frac=0.01, bits=16)
    img[200:400] = np.minimum(img[200:400].astype(np.int64) + 30000, 65535).astype(np.uint16)
    img[500:520, 100:140] = rng.integers(50000, 65536, size=(20, 40))
    d, p = pair(4.0, hmf=(7, 5, 3))
    ref = oracle.extract(img, d)
    assert ref.sum() > 0
    assert_same(run(cuda_lib, img, p), ref, "full range, hmf 7 5 3")

