"""FP64 CPU oracle for the feature-extraction path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports,
links or executes it, and the two share no code: the oracle is plain C
(``fx_oracle.c``) plus the independent pure-Python brute force in
``brute.py``; neither imports the CUDA package.

The method (arXiv 1304.3992): two 5x5 LoG masks (Eq. 1, Sec. 4.1), zero
crossings with a contrast threshold (Sec. 3.2), the 5x5 / 3x3 standard
deviation test (Eq. 2, Sec. 4.1), OR-combination (Sec. 4.1) and the hybrid
median filter (Sec. 3.4, repeated per Sec. 4.2).  The readings taken where the
paper is silent are listed at the top of ``fx_oracle.c``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, exhaustive brute force, and the independent
``brute.py``).  Agreement with the paper's own output figures is unpinned:
the figures and the datasets are absent from the paper's text.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfx_oracle.so")

# Layout of the parameter vector handed to fxo_extract (mirrors the enum in
# fx_oracle.c).
PARAM_ORDER = (
    "sigma1", "sigma2", "mask_q", "t_zc1", "t_zc2", "t_sd5_1", "t_sd5_2",
    "t_sdmax_1", "t_sdmax_2", "t_sd3_1", "t_sd3_2", "stddev_source",
    "hmf0", "hmf1", "hmf2", "hmf3", "log_mode",
)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fx_oracle.c into a shared library with gcc (no fast-math, no FMA
    contraction, so x86 and Arm hosts evaluate Eq. 1 identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.fxo_log_mask.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
            lib.fxo_log_mask.restype = ctypes.c_int
            lib.fxo_log_mask_fp32.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            lib.fxo_log_mask_fp32.restype = ctypes.c_int
            lib.fxo_extract.argtypes = [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                ctypes.c_longlong, dp, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                ctypes.c_void_p, ctypes.c_void_p,
            ]
            lib.fxo_extract.restype = ctypes.c_int
            lib.fxo_hybrid_median.argtypes = [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p,
            ]
            lib.fxo_hybrid_median.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_params(scale: float = 1.0) -> dict:
    """Threshold proposals of the design notes (the paper prints none): a
    12 DN step on 8-bit data, times the value scale (1, 8 or 16)."""
    return dict(
        sigma=(0.5, 20.0), mask_q=512,
        t_zc=(4248.0 * scale, 15360.0 * scale),
        t_sd5=(6.0 * scale, 6.0 * scale), t_sdmax=(24.0 * scale, 24.0 * scale),
        t_sd3=(6.0 * scale, 6.0 * scale),
        stddev_source=0, hmf=(5,), log_mode=0,
    )


def _param_vector(p: dict) -> np.ndarray:
    hmf = p.get("hmf", (5,))
    if isinstance(hmf, int):
        hmf = (hmf,) if hmf else ()
    hmf = tuple(hmf) + (0,) * (4 - len(hmf))
    v = [
        p["sigma"][0], p["sigma"][1], p["mask_q"], p["t_zc"][0], p["t_zc"][1],
        p["t_sd5"][0], p["t_sd5"][1], p["t_sdmax"][0], p["t_sdmax"][1],
        p["t_sd3"][0], p["t_sd3"][1], p.get("stddev_source", 0), *hmf, p.get("log_mode", 0),
    ]
    return np.ascontiguousarray(np.array(v, dtype=np.float64))


def log_mask(sigma: float, q: float = 512):
    """Reading R1: returns (samples of Eq. 1, integer mask), both 5x5 float64."""
    g = np.zeros(25)
    w = np.zeros(25)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().fxo_log_mask(float(sigma), float(q), g.ctypes.data_as(dp), w.ctypes.data_as(dp))
    if rc != 0:
        raise ValueError(f"fxo_log_mask rc={rc}")
    return g.reshape(5, 5), w.reshape(5, 5)


def log_mask_fp32(sigma: float, q: float = 512) -> np.ndarray:
    """Reading R9: the FP32-LoG mode's mask (5x5 float64, exact grid values)."""
    w = np.zeros(25)
    rc = _load().fxo_log_mask_fp32(float(sigma), float(q), w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError(f"fxo_log_mask_fp32 rc={rc}")
    return w.reshape(5, 5)


STAGE_NAMES = ("L1", "L2", "Z1", "Z2", "C1", "C2", "S1", "S2", "M")


def extract(img: np.ndarray, params: dict, rows=None, stages: bool = False):
    """Extraction mask (uint8 0/1) of a 2-D uint8/uint16 image.

    ``img`` may be a strided view whose rows are contiguous (pitched buffer).
    ``rows=(y0, y1)`` computes only those output rows (the full image still
    defines the borders).  With ``stages=True`` also returns a dict of the
    intermediate planes for the same rows."""
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16) or img.strides[1] != img.itemsize:
        raise ValueError("img must be a 2-D uint8/uint16 array with contiguous rows")
    H, W = img.shape
    y0, y1 = (0, H) if rows is None else rows
    out = np.zeros((y1 - y0, W), dtype=np.uint8)
    st = np.zeros((9, y1 - y0, W), dtype=np.float64) if stages else None
    prm = _param_vector(params)
    rc = _load().fxo_extract(
        img.ctypes.data, img.itemsize, W, H, img.strides[0],
        prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), prm.size, y0, y1,
        out.ctypes.data, st.ctypes.data if st is not None else None)
    if rc != 0:
        raise ValueError(f"fxo_extract rc={rc}")
    if stages:
        return out, {n: st[i] for i, n in enumerate(STAGE_NAMES)}
    return out


def hybrid_median(img: np.ndarray, window: int = 5) -> np.ndarray:
    """Grayscale hybrid median (Sec. 3.4, reading R6) of a uint8/uint16 image."""
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16) or img.strides[1] != img.itemsize:
        raise ValueError("img must be a 2-D uint8/uint16 array with contiguous rows")
    H, W = img.shape
    out = np.zeros((H, W), dtype=np.uint16)
    rc = _load().fxo_hybrid_median(img.ctypes.data, img.itemsize, W, H, img.strides[0],
                                   int(window), out.ctypes.data)
    if rc != 0:
        raise ValueError(f"fxo_hybrid_median rc={rc}")
    return out.astype(img.dtype)
