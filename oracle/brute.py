"""Second, independent oracle: pure-Python per-pixel definitions -- TEST
INFRASTRUCTURE ONLY (tiny images; used by ``tests/`` to cross-check the C
oracle).

Where ``fx_oracle.c`` runs one pass per stage over arrays, this module writes
each quantity of the method as a function of one pixel, evaluated on demand
with Python integers and exact rationals:

* ``L(f, x, y)``  Eq. 1 mask applied to the 5x5 neighbourhood (Sec. 4.1);
                  integer masks, or the FP32-LoG mode's grid masks as exact
                  rationals
* ``Z(f, x, y)``  zero crossing among the 4 neighbours (Sec. 3.2)
* ``C(f, x, y)``  contrast max - min over the pixel and its 4 neighbours (Sec. 3.2)
* ``S(f, x, y)``  standard deviation of Eq. 2 with exact rationals (Sec. 4.1)
* ``M(x, y)``     OR of the two extracted maps (Sec. 4.1)
* ``H(i, x, y)``  hybrid median, level i (Sec. 3.4)

Every stage reads its predecessor at clamped coordinates (replicated borders).
The mask construction repeats the reading of Eq. 1 (mean removal, scale to
max |w| = Q, round half away from zero, centre reset) in its own code.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache


def _centred_samples(sigma: float):
    samples = {}
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            r2 = dx * dx + dy * dy
            s2 = sigma * sigma
            samples[(dx, dy)] = (-1.0 / (math.pi * s2 * s2) * (1.0 - r2 / (2.0 * s2))
                                 * math.exp(-r2 / (2.0 * s2)))
    acc = 0.0
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            acc += samples[(dx, dy)]
    mean = acc / 25.0
    centred = {k: v - mean for k, v in samples.items()}
    return centred, max(abs(v) for v in centred.values())


def log_mask_fp32(sigma: float, q: float):
    """FP32-LoG mode: the centred samples scaled to max |w| = q, rounded half
    away from zero to multiples of 2^(e-23) (2^e the smallest power of two >= q),
    centre reset to minus the sum of the others.  Returns dict (dx,dy)->Fraction."""
    centred, biggest = _centred_samples(sigma)
    e = 0
    while 2 ** e < q:
        e += 1
    grid = Fraction(2) ** (e - 23)
    w = {}
    for k, v in centred.items():
        t = q * v / biggest / float(grid)
        m = int(math.floor(t + 0.5)) if t >= 0 else -int(math.floor(-t + 0.5))
        w[k] = m * grid
    w[(0, 0)] = -sum(v for k, v in w.items() if k != (0, 0))
    return w


def log_mask(sigma: float, q: float):
    """Eq. 1 on the 5x5 grid, made zero-sum and integer (returns dict (dx,dy)->int)."""
    samples = {}
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            r2 = dx * dx + dy * dy
            s2 = sigma * sigma
            samples[(dx, dy)] = (-1.0 / (math.pi * s2 * s2) * (1.0 - r2 / (2.0 * s2))
                                 * math.exp(-r2 / (2.0 * s2)))
    # fx_oracle.c sums in row order without compensation; use the same order so
    # both oracles see the identical double (a compensated sum could differ in
    # the last bit, which only matters at an exact rounding tie)
    acc = 0.0
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            acc += samples[(dx, dy)]
    mean = acc / 25.0
    centred = {k: v - mean for k, v in samples.items()}
    biggest = max(abs(v) for v in centred.values())
    w = {}
    for k, v in centred.items():
        t = q * v / biggest
        w[k] = int(math.floor(t + 0.5)) if t >= 0 else -int(math.floor(-t + 0.5))
    w[(0, 0)] = -sum(v for k, v in w.items() if k != (0, 0))
    return w


class Brute:
    def __init__(self, img, params):
        """img: list of rows (lists of ints). params: the dict used by oracle.extract."""
        self.img = img
        self.height = len(img)
        self.width = len(img[0])
        self.p = params
        make = log_mask_fp32 if params.get("log_mode", 0) == 1 else log_mask
        self.w = [make(params["sigma"][f], params["mask_q"]) for f in range(2)]
        hmf = params.get("hmf", (5,))
        if isinstance(hmf, int):
            hmf = (hmf,) if hmf else ()
        self.hmf = tuple(hmf)
        self.source = params.get("stddev_source", 0)
        self._L = lru_cache(maxsize=None)(self._L_raw)
        self._Z = lru_cache(maxsize=None)(self._Z_raw)
        self._M = lru_cache(maxsize=None)(self._M_raw)
        self._H = lru_cache(maxsize=None)(self._H_raw)

    def clamp(self, x, y):
        return min(max(x, 0), self.width - 1), min(max(y, 0), self.height - 1)

    def I(self, x, y):
        x, y = self.clamp(x, y)
        return int(self.img[y][x])

    def L(self, f, x, y):
        return self._L(f, *self.clamp(x, y))

    def _L_raw(self, f, x, y):
        return sum(wv * self.I(x + dx, y + dy) for (dx, dy), wv in self.w[f].items())

    def Z(self, f, x, y):
        return self._Z(f, *self.clamp(x, y))

    def _Z_raw(self, f, x, y):
        v = self.L(f, x, y)
        west, east = self.L(f, x - 1, y), self.L(f, x + 1, y)
        north, south = self.L(f, x, y - 1), self.L(f, x, y + 1)
        if v == 0:
            return int((west < 0 < east) or (east < 0 < west)
                       or (north < 0 < south) or (south < 0 < north))
        opposite = [q for q in (west, east, north, south) if (q < 0 < v) or (v < 0 < q)]
        if not opposite:
            return 0
        # smallest absolute value among the opposite-signed pairs; an exact
        # tie is given to the negative pixel
        for q in opposite:
            if abs(v) > abs(q) or (abs(v) == abs(q) and v > 0):
                return 0
        return 1

    def C(self, f, x, y):
        x, y = self.clamp(x, y)
        vals = [self.L(f, x, y), self.L(f, x - 1, y), self.L(f, x + 1, y),
                self.L(f, x, y - 1), self.L(f, x, y + 1)]
        return int(max(vals) - min(vals) > self.p["t_zc"][f])

    def _window(self, f, x, y, r):
        if self.source == 0:
            return [self.I(x + dx, y + dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
        return [self.Z(f, x + dx, y + dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]

    @staticmethod
    def _sd_exceeds(vals, t):
        """Eq. 2 with exact rationals: unbiased s > t."""
        if t < 0:
            return True
        n = len(vals)
        mean = Fraction(sum(vals), n)
        var = sum((Fraction(a) - mean) ** 2 for a in vals) / (n - 1)
        return var > Fraction(t) ** 2

    def S(self, f, x, y):
        x, y = self.clamp(x, y)
        w5 = self._window(f, x, y, 2)
        if self._sd_exceeds(w5, self.p["t_sdmax"][f]):
            return int(self._sd_exceeds(self._window(f, x, y, 1), self.p["t_sd3"][f]))
        return int(self._sd_exceeds(w5, self.p["t_sd5"][f]))

    def E(self, f, x, y):
        return int(self.Z(f, x, y) and self.C(f, x, y) and self.S(f, x, y))

    def M(self, x, y):
        return self._M(*self.clamp(x, y))

    def _M_raw(self, x, y):
        return int(self.E(0, x, y) or self.E(1, x, y))

    def H(self, level, x, y):
        """Output after `level` hybrid-median passes (level 0 = combined map)."""
        if level == 0:
            return self.M(x, y)
        return self._H(level, *self.clamp(x, y))

    def _H_raw(self, level, x, y):
        k = self.hmf[level - 1]
        r = k // 2
        prev = lambda a, b: self.H(level - 1, a, b)
        plus = [prev(x + d, y) for d in range(-r, r + 1)] + \
               [prev(x, y + d) for d in range(-r, r + 1) if d != 0]
        cross = [prev(x + d, y + d) for d in range(-r, r + 1)] + \
                [prev(x + d, y - d) for d in range(-r, r + 1) if d != 0]
        med = lambda v: sorted(v)[len(v) // 2]
        return med([med(plus), med(cross), prev(x, y)])

    def output(self):
        lv = len(self.hmf)
        return [[self.H(lv, x, y) for x in range(self.width)] for y in range(self.height)]
