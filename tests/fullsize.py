"""Row bands of the full-size parity tests.

fx_extract splits an image into work units of uh output rows (a warp walks a
strip of 56, 52, 44 or 36 output columns over uh rows); a unit starts its rows with a prefill and ends
with the rows its outputs need, and its 16-row bit blocks restart at each
unit.  The bands compared with the oracle therefore straddle unit seams on
purpose.  unit_height() restates the launch's wave model (rows walked x waves
of resident warps, minimised over heights that are multiples of 16 up to 768)
so the tests can place bands on the seams of the launch they check.
"""
from __future__ import annotations

import numpy as np

FIRST_PASS_CTAS = 13  # one-warp CTAs per SM of the streaming first pass
WARPS_PER_CTA = 1


def strip_width(r_m: int, source: int = 0) -> int:
    """Output columns of the streaming strip class serving median radius sum
    r_m: 64 minus twice the halo (3 + the class radius 1, 3, 7 or 11, plus 2
    for the crossing-map source)."""
    rc = 1 if r_m <= 1 else 3 if r_m <= 3 else 7 if r_m <= 7 else 11
    return 58 - 2 * rc - (4 if source == 1 else 0)


def unit_height(rows: int, width: int, sms: int, r_m: int = 2, source: int = 0) -> int:
    units_x = -(-width // strip_width(r_m, source))
    slots = sms * FIRST_PASS_CTAS * WARPS_PER_CTA
    overhead = 20 + r_m + (2 if source == 1 else 0)
    best, best_cost = 768, None
    for uh in range(768, 15, -16):
        cost = -(-units_x * (-(-rows // uh)) // slots) * (uh + overhead)
        if best_cost is None or cost < best_cost:
            best, best_cost = uh, cost
    return best


def seam_bands(H: int, uh: int, seams: int = 3, half: int = 20, edge: int = 24, seed: int = 0):
    """Bands of 2*half rows centred on the first `seams` unit seams, the first
    and last `edge` rows, and one band at a seeded random position."""
    bands = [(0, edge), (H - edge, H)]
    for k in range(1, seams + 1):
        y = k * uh
        if y + half <= H:
            bands.append((y - half, y + half))
    rng = np.random.default_rng(seed)
    y = int(rng.integers(edge, H - edge - 2 * half))
    bands.append((y, y + 2 * half))
    return bands
