"""Writes tests/golden/pan512_u8_digest.txt from the oracle alone.

The digest (SHA-256 of the 512 x 512 extraction mask of the seeded PAN scene,
plus per-row counts) is a regression pin: it changes only when the oracle's
arithmetic or the scene generator changes, which a commit must then justify.
Run: python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from gen import scenes  # noqa: E402


def digest_lines():
    img = scenes.pan_512_u8()
    mask = oracle.extract(img, oracle.default_params(1.0))
    lines = [
        "# oracle mask of gen.scenes.pan_512_u8() with oracle.default_params(1.0)",
        f"sha256 {hashlib.sha256(mask.tobytes()).hexdigest()}",
        f"ones {int(mask.sum())}",
        "row_counts " + " ".join(str(int(c)) for c in mask.sum(axis=1)),
    ]
    return lines


if __name__ == "__main__":
    with open(os.path.join(HERE, "pan512_u8_digest.txt"), "w") as f:
        f.write("\n".join(digest_lines()) + "\n")
