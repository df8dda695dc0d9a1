"""CPU model of the streaming first pass's row loads (Strip::run and step in
csrc/fx_stream.cuh): every row a unit loads lies in the rows its buffer holds.

A unit of output rows [Y0, Y1) prefills its rings from row Y0 + 4 kK0 (kK0 =
-2 on the compact and narrow strips, -3 on the wide, -4 on the extra-wide
ones), then runs four steps per iteration k, each loading the row la ahead (la
= 7 through the cp.async ring, 4 through registers).  Loads clamp to the
buffer's rows [rlo, rhi] (relative to Y0) except in the unchecked body, which
runs only when every row the iteration loads lies there; load offsets count
from rbase = max(rlo, 4 kK0) and must not be negative.  The model walks that
schedule, tail skip included, for image heights, unit heights, median lists,
both deviation sources and row windows (the buffer holding the window plus the
input radius r_in = r_m + 3 (+2) of the host's row bands, or a wider margin),
and counts loads that would leave the buffer.
"""
import pytest


def k0_of(r_m: int) -> int:
    return -2 if r_m <= 3 else -3 if r_m <= 7 else -4


def out_of_buffer_loads(H, row0, row_lim, y_begin, y_end, uh, nhmf, src_z, r_m, ring, tail):
    k0 = k0_of(r_m)
    la = 7 if ring else 4
    bad = 0
    for Y0 in range(y_begin, y_end, uh):
        Y1 = min(Y0 + uh, y_end)
        rlo, rhi = max(row0, 0) - Y0, min(row_lim, H) - 1 - Y0
        rbase = max(rlo, 4 * k0)
        Hrel, Y0rel = H - Y0, min(Y0, 1 << 30)
        iters = 4 * ((Y1 - Y0 + 2) // 16 + 2 + max(nhmf, 1) + (1 if src_z else 0))
        t_end = (Y1 - Y0 - 1) + r_m + 4 + (2 if src_z else 0)

        def load(t, clamp):
            yr = min(max(t, rlo), rhi) if clamp else t
            return 0 if (rlo <= yr <= rhi and yr - rbase >= 0) else 1

        for i in range(la):  # prefill, clamped
            bad += load(4 * k0 + i, True)
        for k in range(k0, iters):
            if tail and 4 * k > t_end:
                continue
            # a strip that is not on the image border: the unchecked body is
            # chosen whenever the row tests allow it
            chk = (4 * k - 2 <= -Y0rel <= 4 * k + 1) or 4 * k + 1 >= Hrel or 4 * k + la < rlo or \
                4 * k + 3 + la > rhi
            for t in range(4 * k, 4 * k + 4):
                bad += load(t + la, chk)
    return bad


LISTS = [  # (median levels, radius sum, crossing-map source)
    (0, 0, False), (1, 1, False), (1, 2, False), (2, 3, False), (1, 2, True), (3, 3, False),
    (2, 4, False), (3, 6, False), (4, 7, True), (3, 9, False), (4, 11, False), (4, 11, True), (3, 8, True),
]


@pytest.mark.parametrize("nhmf,r_m,src_z", LISTS)
def test_no_load_leaves_the_buffer(nhmf, r_m, src_z):
    r_in = r_m + 3 + (2 if src_z else 0)
    bad = 0
    for H in [1, 2, 5, 17, 33, 100, 257, 700, 1000, 2049]:
        for uh in [16, 48, 128, 512, 656, 752]:
            for ring in (False, True):
                for tail in (False, True):
                    bad += out_of_buffer_loads(H, 0, H, 0, H, uh, nhmf, src_z, r_m, ring, tail)
                    for y0, y1 in [(0, min(H, 64)), (H // 3, min(H, H // 3 + 70)), (max(0, H - 40), H)]:
                        if y1 <= y0 or (0 < y0 < 19):  # row windows start at row 0 or >= 19
                            continue
                        for margin in (r_in, r_in + 4):
                            a, b = max(0, y0 - margin), min(H, y1 + margin)
                            bad += out_of_buffer_loads(H, a, b, y0, y1, uh, nhmf, src_z, r_m, ring, tail)
    assert bad == 0


def test_the_model_sees_an_unclamped_load():
    """The model is not vacuous: with the row tests of the unchecked body
    dropped (every iteration unchecked), loads leave a buffer that starts at
    the row window."""
    H, a, b, y0, y1 = 300, 100 - 6, 170 + 6, 100, 170
    k0, la = k0_of(3), 7
    rlo, rhi = a - y0, b - 1 - y0
    rbase = max(rlo, 4 * k0)
    bad = 0
    for k in range(k0, 4 * ((y1 - y0 + 2) // 16 + 3)):
        for t in range(4 * k, 4 * k + 4):
            yr = t + la
            bad += 0 if (rlo <= yr <= rhi and yr - rbase >= 0) else 1
    assert bad > 0
