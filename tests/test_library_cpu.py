"""CPU-only checks of the C-ABI library: it loads, exports every entry point
declared in include/fx.h, and its host-side logic (defaults, the integer
masks, argument validation that fails before any device call) is right.
No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fx():
    from paper_1304_3992_gb300 import build, fx as b
    build.build()
    b.load()
    return b


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "fx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(fx_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_entry_points_are_exported(fx):
    names = _declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(fx.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fx.exported_names())


def test_version(fx):
    assert fx.load().fx_version().startswith(b"fx ")


@pytest.mark.parametrize("sigma", [0.5, 20.0, 0.8, 1.3, 3.3, 100.0])
@pytest.mark.parametrize("q", [64, 512, 2000])
def test_library_mask_equals_oracle(fx, sigma, q):
    """The library's own construction of the Eq. 1 masks matches the oracle's."""
    _, w = oracle.log_mask(sigma, q)
    assert np.array_equal(np.array(fx.log_mask(sigma, q)), w.astype(int))


def test_defaults(fx):
    p8 = fx.make_params(fx.FX_U8)
    assert list(p8.sigma) == [0.5, 20.0] and p8.mask_q == 512 and list(p8.hmf) == [5, 0, 0, 0]
    assert list(p8.t_zc) == [4248.0, 15360.0] and list(p8.t_sd5) == [6.0, 6.0]
    assert list(p8.t_sdmax) == [24.0, 24.0] and list(p8.t_sd3) == [6.0, 6.0]
    p16 = fx.make_params(fx.FX_U16)
    assert p16.bits == 12 and list(p16.t_zc) == [4248.0 * 16, 15360.0 * 16]
    p11 = fx.make_params(fx.FX_U16, 11)
    assert list(p11.t_sdmax) == [24.0 * 8, 24.0 * 8]
    ref = oracle.default_params(16.0)
    assert tuple(p16.t_zc) == ref["t_zc"] and tuple(p16.t_sd5) == ref["t_sd5"]


def test_invalid_arguments_rejected_before_any_device_call(fx):
    lib = fx.load()
    p = fx.make_params(fx.FX_U16)
    bad = [
        (0, 8, 8, 16, fx.FX_U16, 4096),        # null image
        (4096, 8, 8, 16, fx.FX_U16, 0),        # null output
        (4096, 0, 8, 16, fx.FX_U16, 8192),     # zero width
        (4096, 8, 0, 16, fx.FX_U16, 8192),     # zero height
        (4096, 8, 8, 15, fx.FX_U16, 8192),     # pitch < width * elem
        (4096, 8, 8, 17, fx.FX_U16, 8192),     # pitch not a multiple of elem
        (4097, 8, 8, 16, fx.FX_U16, 8192),     # misaligned uint16 image
        (4096, 8, 8, 16, 3, 8192),             # bad dtype
        (4096, 8, 8, 16, fx.FX_U16, 4100),     # output overlaps the image
    ]
    for img, w, h, pitch, dt, out in bad:
        assert lib.fx_extract(img, w, h, pitch, dt, ctypes.byref(p), out, None) == 1, (img, w, h, pitch, dt, out)
    q = fx.make_params(fx.FX_U16)
    q.struct_size = 7
    assert lib.fx_extract(4096, 8, 8, 16, fx.FX_U16, ctypes.byref(q), 1 << 20, None) == 1


def test_specialize_argument_checks(fx):
    """fx_specialize validates before touching a device or the run-time
    compiler: null parameters, a wrong struct size or dtype are rejected,
    parameters that overflow the exact evaluation return FX_ERR_RANGE, and
    median lists beyond the streaming kernel are not specialised."""
    lib = fx.load()
    p = fx.make_params(fx.FX_U16, 12)
    assert lib.fx_specialize(None, fx.FX_U16) == 1
    assert lib.fx_specialize(ctypes.byref(p), 3) == 1
    q = fx.make_params(fx.FX_U16, 12)
    q.struct_size = 7
    assert lib.fx_specialize(ctypes.byref(q), fx.FX_U16) == 1
    big = fx.make_params(fx.FX_U16, 16, mask_q=1 << 19)
    assert lib.fx_specialize(ctypes.byref(big), fx.FX_U16) == 3
    assert lib.fx_specialize(ctypes.byref(fx.make_params(fx.FX_U16, 12, hmf=(7, 7, 7, 7))), fx.FX_U16) == 2


def test_plan_argument_checks(fx):
    lib = fx.load()
    h = ctypes.c_void_p()
    p = fx.make_params(fx.FX_U16)
    assert lib.fx_plan_create(None, ctypes.byref(p), 4, 0) == 1
    assert lib.fx_plan_create(ctypes.byref(h), ctypes.byref(p), 0, 0) == 1
    assert lib.fx_plan_destroy(None) == 1
    assert lib.fx_extract_batch(None, None, 1, None) == 1
    assert lib.fx_get_device_status(None, None) == 1
    assert lib.fx_status_string(3) == b"FX_ERR_RANGE"
