"""Seeded synthetic single-band scenes shaped like panchromatic and
multispectral satellite data.

The paper's Cartosat-1 PAN and Resourcesat-2 AWiFS scenes (Sec. 6) are not
available, so these seeded scenes stand in for them with the same bit depths
(8-bit PAN, 11/12-bit multispectral) and the structure the method looks for:
a smooth low-frequency background, sharp-edged man-made blocks (buildings,
water bodies), sensor noise and salt-and-pepper impulses.

This module holds none of the extraction method's arithmetic.  Both the
oracle tests and the CUDA tests / benchmark draw their inputs here.

Recipe (``numpy.random.default_rng(seed)``, PCG64; draws in this order):

1. Background: 4 isotropic Gaussians; per Gaussian the centre (x then y)
   uniform over the image, sigma uniform in [side/8, side/2] with
   side = (W+H)/2, amplitude uniform in [0.5, 1].  The sum is affinely
   rescaled to [60, 180] DN (8-bit scale).
2. Rectangles, painted in order; per rectangle: centre x, centre y (uniform
   over the image), two sides uniform in [8, 60] px, a rotation flag
   (probability 1/2), an angle uniform in [0, pi) (drawn always, used only
   when rotated), a value uniform in the integers 80..250.  A pixel belongs to
   the rectangle when its centre (integer coordinates) lies in
   [-a/2, a/2) x [-b/2, b/2) of the rectangle's own frame.
3. Band: clean * gain * scale plus N(0, noise_sigma^2) noise drawn with the
   band's own noise generator (float32 standard normals), rounded half to
   even and clipped to [0, 2^bits - 1].
4. Impulses: n = round(rho * W * H) positions drawn uniformly (with
   replacement) from the same noise generator, then one fair bit per position
   chooses pepper (0) or salt (2^bits - 1).
"""
from __future__ import annotations

import math

import numpy as np


def clean_scene(width: int, height: int, rng: np.random.Generator, n_rects: int) -> np.ndarray:
    """Steps 1-2 of the recipe: float32 scene in 8-bit DN."""
    W, H = int(width), int(height)
    side = 0.5 * (W + H)
    xs = np.arange(W, dtype=np.float32)
    ys = np.arange(H, dtype=np.float32)
    img = np.zeros((H, W), dtype=np.float32)
    for _ in range(4):
        cx = rng.uniform(0, W)
        cy = rng.uniform(0, H)
        s = rng.uniform(side / 8, side / 2)
        amp = rng.uniform(0.5, 1.0)
        gx = np.exp(-((xs - np.float32(cx)) ** 2) / np.float32(2 * s * s)).astype(np.float32)
        gy = np.exp(-((ys - np.float32(cy)) ** 2) / np.float32(2 * s * s)).astype(np.float32)
        img += np.float32(amp) * gy[:, None] * gx[None, :]
    lo, hi = float(img.min()), float(img.max())
    if hi > lo:
        img -= np.float32(lo)
        img *= np.float32(120.0 / (hi - lo))
        img += np.float32(60.0)
    else:
        img[:] = 120.0
    for _ in range(n_rects):
        cx = rng.uniform(0, W)
        cy = rng.uniform(0, H)
        a = rng.uniform(8, 60)
        b = rng.uniform(8, 60)
        rotated = rng.random() < 0.5
        theta = rng.uniform(0, math.pi)
        val = int(rng.integers(80, 251))
        if not rotated:
            theta = 0.0
        r = 0.5 * math.hypot(a, b) + 1
        x0, x1 = max(0, int(math.floor(cx - r))), min(W, int(math.ceil(cx + r)) + 1)
        y0, y1 = max(0, int(math.floor(cy - r))), min(H, int(math.ceil(cy + r)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        px = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
        py = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
        c, s_ = math.cos(theta), math.sin(theta)
        u = c * px + s_ * py
        v = -s_ * px + c * py
        inside = (u >= -a / 2) & (u < a / 2) & (v >= -b / 2) & (v < b / 2)
        img[y0:y1, x0:x1][inside] = val
    return img


def band(clean: np.ndarray, *, gain: float, scale: float, noise_sigma: float,
         impulse_frac: float, noise_seed: int, bits: int) -> np.ndarray:
    """Steps 3-4 of the recipe: one noisy band as uint8 (bits <= 8) or uint16."""
    rng = np.random.default_rng(noise_seed)
    maxval = (1 << bits) - 1
    H, W = clean.shape
    out_dtype = np.uint8 if bits <= 8 else np.uint16
    v = clean * np.float32(gain * scale)
    v += rng.standard_normal(size=clean.shape, dtype=np.float32) * np.float32(noise_sigma)
    np.rint(v, out=v)
    np.clip(v, 0, maxval, out=v)
    img = v.astype(out_dtype)
    del v
    n = int(round(impulse_frac * W * H))
    if n:
        pos = rng.integers(0, W * H, size=n)
        salt = rng.integers(0, 2, size=n).astype(bool)
        flat = img.reshape(-1)
        flat[pos[salt]] = maxval
        flat[pos[~salt]] = 0
    return img


def scene(width: int, height: int, *, seed: int, n_rects: int, noise_sigma: float,
          impulse_frac: float, bits: int, gain: float = 1.0, noise_seed: int | None = None) -> np.ndarray:
    """One single-band scene; the value scale is 2^(bits-8) (1, 8, 16 for 8, 11, 12 bits)."""
    rng = np.random.default_rng(seed)
    clean = clean_scene(width, height, rng, n_rects)
    scale = float(1 << (bits - 8)) if bits > 8 else 1.0
    return band(clean, gain=gain, scale=scale, noise_sigma=noise_sigma, impulse_frac=impulse_frac,
                noise_seed=seed + 1_000_003 if noise_seed is None else noise_seed, bits=bits)


# --------------------------------------------------------------- workloads

def pan_512_u8() -> np.ndarray:
    """512 x 512 uint8 panchromatic scene, seed 0: 40 rectangles, noise sigma 4, 1 % impulses."""
    return scene(512, 512, seed=0, n_rects=40, noise_sigma=4.0, impulse_frac=0.01, bits=8)


def ms_8192_u16_11bit() -> np.ndarray:
    """8192 x 8192 uint16 scene of 11-bit values, seed 1: 4000 rectangles,
    noise sigma 12, 0.5 % impulses."""
    return scene(8192, 8192, seed=1, n_rects=4000, noise_sigma=12.0, impulse_frac=0.005, bits=11)


def ms_bands_u16_12bit(side: int = 16384, n_bands: int = 4, n_rects: int = 16000,
                       bands=None):
    """Multispectral scene: n_bands x side^2 uint16, 12-bit.  Shared geometry
    (seed 2); per-band gain uniform in [0.7, 1.3] drawn from the geometry
    generator after the rectangles; noise seeds 3, 4, 5, 6; noise sigma 24;
    0.5 % impulses.  Yields the bands one at a time (``bands`` selects)."""
    rng = np.random.default_rng(2)
    clean = clean_scene(side, side, rng, n_rects)
    gains = [rng.uniform(0.7, 1.3) for _ in range(n_bands)]
    for b in range(n_bands) if bands is None else bands:
        yield band(clean, gain=gains[b], scale=16.0, noise_sigma=24.0, impulse_frac=0.005,
                   noise_seed=3 + b, bits=12)


def uneven_batch(n: int = 64, lo: int = 1000, hi: int = 12000, seed: int = 100,
                 master_side: int = 12000):
    """Batch of n single-band scenes of uneven size: sides uniform in [lo, hi]
    (widths redrawn while a multiple of 32), uint8 for even i and 12-bit
    uint16 for odd i, row pitch rounded up to 256 B.  To keep generation cheap
    the scenes are crops at uniform offsets of two master scenes (uint8 and
    uint16) of the same recipe (rectangle density of the 512^2 PAN scene).

    Returns a list of (img_view, pitched_buffer) with img_view a strided
    (h, w) view into a (h, pitch/elem) buffer."""
    rng = np.random.default_rng(seed)
    dens = 40 / (512 * 512)
    nr = int(round(dens * master_side * master_side))
    m8 = scene(master_side, master_side, seed=seed + 1, n_rects=nr, noise_sigma=4.0,
               impulse_frac=0.01, bits=8)
    m16 = scene(master_side, master_side, seed=seed + 2, n_rects=nr, noise_sigma=24.0,
                impulse_frac=0.005, bits=12)
    out = []
    for i in range(n):
        w = int(rng.integers(lo, hi + 1))
        while w % 32 == 0:
            w = int(rng.integers(lo, hi + 1))
        h = int(rng.integers(lo, hi + 1))
        master = m8 if i % 2 == 0 else m16
        w, h = min(w, master.shape[1]), min(h, master.shape[0])
        ox = int(rng.integers(0, master.shape[1] - w + 1))
        oy = int(rng.integers(0, master.shape[0] - h + 1))
        elem = master.itemsize
        pitch = ((w * elem + 255) // 256) * 256
        buf = np.zeros((h, pitch // elem), dtype=master.dtype)
        buf[:, :w] = master[oy:oy + h, ox:ox + w]
        out.append((buf[:, :w], buf))
    return out


def pitched(img: np.ndarray, pitch_bytes: int, fill: int = 0) -> np.ndarray:
    """Copy img into a buffer whose rows are pitch_bytes apart; returns the (h, w) view."""
    h, w = img.shape
    assert pitch_bytes % img.itemsize == 0 and pitch_bytes >= w * img.itemsize
    buf = np.full((h, pitch_bytes // img.itemsize), fill, dtype=img.dtype)
    buf[:, :w] = img
    return buf[:, :w]
