"""The allocation-free batched entry point, fx_extract_batch_noalloc.

It exists for callers that may not allocate device memory (their memory is
owned by another allocator or pool, or allocation is forbidden after start-up):
its scratch is a fixed array inside libfx.so.  This file is collected last on
purpose, so that a failure here cannot hide any other test.  The tests call the
entry point through the C ABI and require masks byte-identical to fx_extract's
(the bar of every mask comparison in this suite), on two calls in a row.
"""
import ctypes

import numpy as np
import pytest

from gen import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _images(seed, n):
    batch = scenes.uneven_batch(n=n, lo=30, hi=500, seed=seed, master_side=600)
    pairs = []
    for view, buf in batch:
        t = torch.from_numpy(buf).cuda()
        img = t[:, :view.shape[1]]
        out = torch.full(view.shape, 7, dtype=torch.uint8, device="cuda")
        pairs.append((img, out))
    return pairs


def _noalloc(fx, params, pairs):
    arr = (fx.ImageDesc * len(pairs))()
    for i, (img, out) in enumerate(pairs):
        arr[i] = fx.desc_for(img, out)
    stream = torch.cuda.current_stream().cuda_stream
    return fx.load().fx_extract_batch_noalloc(ctypes.byref(params), arr, len(pairs), stream)


def test_noalloc_matches_fx_extract_twice(cuda_lib):
    """Calls in a row (the scratch keeps the previous call's counter) give the
    masks of fx_extract.  The 12-bit thresholds exercise the uint16 images, the
    8-bit thresholds of the last call the uint8 ones (their masks are empty
    under 12-bit thresholds), so each pixel type is compared on masks with
    feature pixels."""
    fx = cuda_lib
    p12 = fx.make_params(fx.FX_U16, 12)
    p8 = fx.make_params(fx.FX_U8, 8)
    features = {1: 0, 2: 0}
    for call, (seed, n, p, elem) in enumerate(((3, 9, p12, 2), (4, 5, p12, 2), (5, 7, p8, 1))):
        pairs = _images(seed, n)
        singles = [fx.extract(img, p).cpu().numpy() for img, _ in pairs]
        assert _noalloc(fx, p, pairs) == 0
        torch.cuda.synchronize()
        for i, ((img, out), ref) in enumerate(zip(pairs, singles)):
            got = out.cpu().numpy()
            assert np.array_equal(got, ref), f"call {call} image {i}: {int((got != ref).sum())} bytes differ"
            if img.element_size() == elem:
                features[elem] += int(ref.sum())
    assert features[1] > 0 and features[2] > 0, features


def test_noalloc_rejects_oversized_batch(cuda_lib):
    fx = cuda_lib
    p = fx.make_params(fx.FX_U16, 12)
    img = torch.zeros((4, 4), dtype=torch.uint16, device="cuda")
    outs = [torch.full((4, 4), 5, dtype=torch.uint8, device="cuda") for _ in range(129)]
    pairs = [(img, o) for o in outs]
    assert _noalloc(fx, p, pairs) == 6  # FX_ERR_BUDGET: more than FX_NOALLOC_MAX_IMAGES
    torch.cuda.synchronize()
    assert all(int(o.min()) == 5 for o in outs), "nothing may be written on error"
