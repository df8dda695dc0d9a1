"""The standalone hybrid median filter (Sec. 3.4) on uint8/uint16 values against
the oracle's grayscale hybrid median (itself pinned to numpy medians): every
output value must be equal."""
import numpy as np
import pytest

import oracle
from gen import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("window", [3, 5, 7])
@pytest.mark.parametrize("shape,bits", [((1, 1), 8), ((1, 70), 16), ((53, 1), 8), ((5, 4), 16),
                                        ((97, 130), 8), ((300, 211), 12), ((67, 1000), 16)])
def test_hmf_matches_oracle(cuda_lib, window, shape, bits):
    h, w = shape
    rng = np.random.default_rng(h * 31 + w + window)
    if bits == 16:
        img = rng.integers(0, 65536, size=shape).astype(np.uint16)
    else:
        big = scenes.scene(max(w, 8) + 4, max(h, 8) + 4, seed=h + w, n_rects=5, noise_sigma=4.0 * (1 << (bits - 8)),
                           impulse_frac=0.05, bits=bits)
        img = np.ascontiguousarray(big[:h, :w])
    got = cuda_lib.hybrid_median(torch.from_numpy(img).cuda(), window).cpu().numpy()
    assert np.array_equal(got, oracle.hybrid_median(img, window))


def test_hmf_pitched_and_errors(cuda_lib):
    import ctypes
    img = scenes.scene(150, 90, seed=3, n_rects=8, noise_sigma=24, impulse_frac=0.02, bits=12)
    buf = torch.zeros((90, 256), dtype=torch.uint16, device="cuda")
    buf[:, :150] = torch.from_numpy(img).cuda()
    obuf = torch.full((90, 200), 7, dtype=torch.uint16, device="cuda")
    cuda_lib.hybrid_median(buf[:, :150], 5, out=obuf[:, :150])
    assert np.array_equal(obuf[:, :150].cpu().numpy(), oracle.hybrid_median(img, 5))
    assert (obuf[:, 150:].cpu().numpy() == 7).all()
    lib = cuda_lib.load()
    t = torch.zeros((8, 8), dtype=torch.uint16, device="cuda")
    assert lib.fx_hybrid_median(t.data_ptr(), 8, 8, 16, 2, 4, obuf.data_ptr(), 0, None) == 1
    assert lib.fx_hybrid_median(t.data_ptr(), 8, 8, 16, 2, 9, obuf.data_ptr(), 0, None) == 1
    assert lib.fx_hybrid_median(t.data_ptr(), 8, 8, 16, 2, 5, t.data_ptr(), 0, None) == 1


@pytest.mark.parametrize("window", [3, 5, 7])
@pytest.mark.parametrize("shape,bits", [((777, 1001), 12), ((600, 61), 8), ((257, 123), 16),
                                        ((385, 1000), 16), ((300, 522), 8), ((131, 113), 12), ((140, 1120), 8)])
def test_hmf_multi_unit(cuda_lib, window, shape, bits):
    """Images spanning several 128-row units (the last one a single row for 257
    and 385 rows) and 60-column strips (56 for window 7): odd widths
    (pixel-by-pixel loads, a width one above a strip of either size) and even
    widths (aligned pair loads: the shared-memory load ring for uint16, 1120 =
    20 strips of 56), against the oracle."""
    h, w = shape
    if bits == 16:
        img = np.random.default_rng(w).integers(0, 65536, size=shape).astype(np.uint16)
    else:
        img = scenes.scene(w, h, seed=w + h, n_rects=40, noise_sigma=4.0 * (1 << (bits - 8)),
                           impulse_frac=0.05, bits=bits)
    got = cuda_lib.hybrid_median(torch.from_numpy(img).cuda(), window).cpu().numpy()
    assert np.array_equal(got, oracle.hybrid_median(img, window))


@pytest.mark.parametrize("window", [3, 5, 7])
def test_hmf_unaligned_output_rows(cuda_lib, window):
    """An even-width uint16 image whose output rows are 2 bytes off a 4-byte
    boundary: the lane pairs are written pixel by pixel."""
    img = np.random.default_rng(window).integers(0, 65536, size=(200, 300)).astype(np.uint16)
    obuf = torch.full((200, 301), 5, dtype=torch.uint16, device="cuda")  # 602-byte rows
    cuda_lib.hybrid_median(torch.from_numpy(img).cuda(), window, out=obuf[:, :300])
    assert np.array_equal(obuf[:, :300].cpu().numpy(), oracle.hybrid_median(img, window))
    assert (obuf[:, 300].cpu().numpy() == 5).all()


@pytest.mark.parametrize("window", [3, 5, 7])
def test_hmf_impulses_and_lines(cuda_lib, window):
    """Closed cases of Sec. 3.4's filter on a flat uint16 image: isolated
    impulses vanish, a one-pixel line along a row, a column or a diagonal
    survives (it fills more than half of one subgroup, and the centre), and a
    step edge stays in place; the whole image against the oracle as well."""
    h, w = 90, 130
    img = np.full((h, w), 1000, dtype=np.uint16)
    for y, x in [(10, 10), (40, 77), (70, 20)]:
        img[y, x] = 60000
    img[25, 30:100] = 50000                          # row line
    img[30:80, 60] = 40000                           # column line
    for d in range(20):
        img[45 + d, 90 + d] = 0                      # diagonal line
    img[:, 120:] = 30000                             # step
    got = cuda_lib.hybrid_median(torch.from_numpy(img).cuda(), window).cpu().numpy()
    assert np.array_equal(got, oracle.hybrid_median(img, window))
    for y, x in [(10, 10), (40, 77), (70, 20)]:
        assert got[y, x] == 1000
    assert (got[25, 40:90] == 50000).all() and (got[40:70, 60] == 40000).all()
    assert all(got[45 + d, 90 + d] == 0 for d in range(4, 16))
    assert (got[:, 120:] == 30000).all() and not (got[:, :120] == 30000).any()
