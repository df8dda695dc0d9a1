"""Parity rule of the FP32-LoG mode (non-integer masks, FP32 responses).

The exact oracle and the FP32 evaluation may disagree only at pixels whose
outcome hangs on an exact response that is tiny against the local response
range: a pixel may differ only if, within the radius its output depends on,
some decision site q of either branch has
    |L(q)|,                                   (the sign of L)
    |L(q) + L(q')| for an opposite-signed 4-neighbour q',  (which of the
                                              pair has the smaller magnitude)
    |max - min of L over q and its 4 neighbours - t_zc|   (the contrast test)
below TAU = 1e-5 of the range (max - min) of the exact L over the 5x5 window
at q.  Such pixels are counted, and their number is capped at CAP = 1e-6 of
the pixels compared.

A mask pixel depends on the decisions at sites within Chebyshev radius
r_dep = (sum of the median radii) + 1 (the 4-neighbour crossing) + 2 when the
standard deviation is taken over the crossing map (its 5x5 window).
"""
from __future__ import annotations

import numpy as np

import oracle

TAU = 1e-5
CAP = 1e-6


def _shifts(a: np.ndarray, r: int):
    """All (2r+1)^2 shifted views of a over its edge-replicated padding."""
    p = np.pad(a, r, mode="edge")
    H, W = a.shape
    return [p[r + dy:r + dy + H, r + dx:r + dx + W] for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def fragile_sites(L: np.ndarray, t_zc: float, tau: float = TAU) -> np.ndarray:
    """Decision sites of one branch whose margin is below tau x the 5x5 range."""
    p = np.pad(L, 1, mode="edge")
    H, W = L.shape
    nb = [p[1:H + 1, 0:W], p[1:H + 1, 2:W + 2], p[0:H, 1:W + 1], p[2:H + 2, 1:W + 1]]
    margin = np.abs(L)
    for q in nb:
        opp = L * q < 0
        margin = np.where(opp, np.minimum(margin, np.abs(L + q)), margin)
    mx = np.maximum.reduce([L] + nb)
    mn = np.minimum.reduce([L] + nb)
    margin = np.minimum(margin, np.abs((mx - mn) - t_zc))
    win = _shifts(L, 2)
    rng = np.maximum.reduce(win) - np.minimum.reduce(win)
    return margin < tau * rng


def dilate(mask: np.ndarray, r: int) -> np.ndarray:
    if r <= 0:
        return mask.copy()
    return np.logical_or.reduce(_shifts(mask, r))


def dependency_radius(params: dict) -> int:
    hmf = params.get("hmf", (5,))
    if isinstance(hmf, int):
        hmf = (hmf,) if hmf else ()
    return sum(k // 2 for k in hmf) + 1 + (2 if params.get("stddev_source", 0) == 1 else 0)


def excused_pixels(Ls, t_zcs, r_dep: int, tau: float = TAU) -> np.ndarray:
    fragile = np.zeros(Ls[0].shape, dtype=bool)
    for L, t in zip(Ls, t_zcs):
        fragile |= fragile_sites(L, t, tau)
    return dilate(fragile, r_dep)


def check(got: np.ndarray, exp: np.ndarray, excused: np.ndarray, cap: float = CAP) -> int:
    """Assert the rule for one compared block; returns the number of differing pixels."""
    diff = got != exp
    bad = diff & ~excused
    if bad.any():
        ys, xs = np.nonzero(bad)
        raise AssertionError(f"{int(bad.sum())} unexcused differences, first at row {ys[0]} col {xs[0]}")
    n = int(diff.sum())
    if n > cap * exp.size:
        raise AssertionError(f"{n} differing pixels exceed the cap {cap} x {exp.size}")
    return n


def compare_with_oracle(img: np.ndarray, got_rows: np.ndarray, params: dict, rows=None) -> int:
    """Check the library's FP32-LoG mask for output rows [y0, y1) of img against
    the exact oracle under the rule above; returns the number of differences."""
    H = img.shape[0]
    y0, y1 = (0, H) if rows is None else rows
    r_dep = dependency_radius(params)
    ext = r_dep + 2  # the fragile test at row y looks 2 rows further
    a, b = max(0, y0 - ext), min(H, y1 + ext)
    exp, st = oracle.extract(img, params, rows=(a, b), stages=True)
    excused = excused_pixels([st["L1"], st["L2"]], params["t_zc"], r_dep)
    sl = slice(y0 - a, y1 - a)
    return check(got_rows, exp[sl], excused[sl])


def tiny_log_excused(Ls, tau: float = TAU) -> np.ndarray:
    """The literal rule: pixels whose exact |L| (either branch) is below tau x
    the range of that branch's L over the 5x5 window at the pixel."""
    ex = np.zeros(Ls[0].shape, dtype=bool)
    for L in Ls:
        win = _shifts(L, 2)
        rng = np.maximum.reduce(win) - np.minimum.reduce(win)
        ex |= np.abs(L) < tau * rng
    return ex


def compare_tiny_log_rule(img: np.ndarray, got_rows: np.ndarray, params: dict, rows=None) -> int:
    """The literal FP32 parity rule: differences only at pixels whose exact
    |LoG| is below 1e-5 of the local response range, at most 1e-6 of the
    pixels compared; returns the number of differences."""
    H = img.shape[0]
    y0, y1 = (0, H) if rows is None else rows
    a, b = max(0, y0 - 2), min(H, y1 + 2)
    exp, st = oracle.extract(img, params, rows=(a, b), stages=True)
    excused = tiny_log_excused([st["L1"], st["L2"]])
    sl = slice(y0 - a, y1 - a)
    return check(got_rows, exp[sl], excused[sl])

