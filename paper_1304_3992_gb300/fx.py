"""Python binding of libfx (the C ABI declared in include/fx.h).

Argument marshalling only: every step of the extraction runs in the CUDA
kernels of libfx.so.  Torch tensors supply device memory and streams; their
pointers are passed as plain integers.  There is no CPU fallback: if the
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfx.so")
# the checked build (every kernel memory index range-checked and counted)
CHECKED_LIB_PATH = os.path.join(_HERE, "_build_checked", "libfx_checked.so")

FX_U8, FX_U16 = 1, 2
FX_LOG_INT, FX_LOG_FP32 = 0, 1
MAX_HMF = 4
STATUS = {0: "FX_OK", 1: "FX_ERR_INVALID_ARG", 2: "FX_ERR_UNSUPPORTED", 3: "FX_ERR_RANGE",
          4: "FX_ERR_CUDA", 5: "FX_ERR_NOMEM", 6: "FX_ERR_BUDGET", 7: "FX_ERR_TIMEOUT"}


class FxError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class Params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("sigma", ctypes.c_double * 2),
        ("mask_q", ctypes.c_int32),
        ("t_zc", ctypes.c_double * 2),
        ("t_sd5", ctypes.c_double * 2),
        ("t_sdmax", ctypes.c_double * 2),
        ("t_sd3", ctypes.c_double * 2),
        ("stddev_source", ctypes.c_int32),
        ("hmf", ctypes.c_int32 * MAX_HMF),
        ("bits", ctypes.c_int32),
        ("out_pitch", ctypes.c_int64),
        ("log_mode", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class ImageDesc(ctypes.Structure):
    _fields_ = [
        ("img", ctypes.c_void_p),
        ("width", ctypes.c_int64),
        ("height", ctypes.c_int64),
        ("pitch_bytes", ctypes.c_int64),
        ("dtype", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("out_mask", ctypes.c_void_p),
        ("out_pitch", ctypes.c_int64),
    ]


_lock = threading.Lock()
_lib = None

_SIGNATURES = {
    "fx_params_default": (None, [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int32]),
    "fx_log_mask": (ctypes.c_int, [ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "fx_log_mask_fp32": (ctypes.c_int, [ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    "fx_extract": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int, ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p]),
    "fx_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Params),
                                      ctypes.c_int32, ctypes.c_int32]),
    "fx_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fx_extract_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ImageDesc), ctypes.c_int32,
                                        ctypes.c_void_p]),
    "fx_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ImageDesc), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "fx_plan_set_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "fx_get_device_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fx_extract_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]),
    "fx_extract_host_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ImageDesc), ctypes.c_int32]),
    "fx_extract_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ImageDesc),
                                                ctypes.c_int32, ctypes.c_void_p]),
    "fx_hybrid_median": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p]),
    "fx_checked_violations": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]),
    "fx_specialize": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int]),
    "fx_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fx_version": (ctypes.c_char_p, []),
}


def exported_names():
    """Entry points the binding expects libfx.so to export (all of include/fx.h)."""
    return tuple(_SIGNATURES)


def load(path: str | None = None):
    """Load libfx.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libfx.so not built ({p}); run __graft_entry__.build()")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise FxError(code, where)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.uint8:
        return FX_U8
    if t.dtype == torch.uint16:
        return FX_U16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def make_params(dtype: int = FX_U16, bits: int = 0, **overrides) -> Params:
    """fx_params_default(dtype, bits) with optional overrides.  Accepts the keys
    sigma, mask_q, t_zc, t_sd5, t_sdmax, t_sd3 (pairs), stddev_source,
    hmf (int or sequence of windows), bits, out_pitch, log_mode (FX_LOG_INT
    or FX_LOG_FP32)."""
    p = Params()
    load().fx_params_default(ctypes.byref(p), dtype, bits)
    for k, v in overrides.items():
        if k in ("sigma", "t_zc", "t_sd5", "t_sdmax", "t_sd3"):
            getattr(p, k)[0], getattr(p, k)[1] = float(v[0]), float(v[1])
        elif k == "hmf":
            seq = (v,) if isinstance(v, int) else tuple(v)
            seq = tuple(x for x in seq if x) + (0,) * MAX_HMF
            for i in range(MAX_HMF):
                p.hmf[i] = int(seq[i])
        elif k in ("mask_q", "stddev_source", "bits", "out_pitch", "log_mode"):
            setattr(p, k, int(v))
        else:
            raise KeyError(k)
    return p


def params_from_dict(d: dict, dtype: int = FX_U16) -> Params:
    """Params from the dictionary form used by the tests (same keys as make_params)."""
    return make_params(dtype, 0, **{k: v for k, v in d.items()})


def log_mask(sigma: float, q: int = 512):
    w = (ctypes.c_int32 * 25)()
    _check(load().fx_log_mask(float(sigma), int(q), w), "fx_log_mask")
    return [list(w[i * 5:(i + 1) * 5]) for i in range(5)]


def log_mask_fp32(sigma: float, q: int = 512):
    """The FP32-LoG mode's non-integer mask (5x5 list of floats)."""
    w = (ctypes.c_float * 25)()
    _check(load().fx_log_mask_fp32(float(sigma), int(q), w), "fx_log_mask_fp32")
    return [list(w[i * 5:(i + 1) * 5]) for i in range(5)]


def extract(img, params: Params | None = None, out=None, stream=None):
    """Extraction mask of a 2-D uint8/uint16 CUDA tensor (rows may be pitched)."""
    import torch
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("img must be a 2-D tensor with contiguous rows")
    h, w = img.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.uint8, device=img.device)
    if out.dim() != 2 or out.stride(1) != 1 or tuple(out.shape) != (h, w):
        raise ValueError("out must be (h, w) uint8 with contiguous rows")
    p = params if params is not None else make_params(_dtype_code(img))
    if out.stride(0) != w:
        p = Params.from_buffer_copy(p)
        p.out_pitch = out.stride(0)
    code = load().fx_extract(img.data_ptr(), w, h, img.stride(0) * img.element_size(), _dtype_code(img),
                             ctypes.byref(p), out.data_ptr(), _stream_ptr(stream))
    _check(code, "fx_extract")
    return out


def hybrid_median(img, window: int = 5, out=None, stream=None):
    """Grayscale hybrid median (Sec. 3.4) of a 2-D uint8/uint16 CUDA tensor."""
    import torch
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("img must be a 2-D tensor with contiguous rows")
    h, w = img.shape
    if out is None:
        out = torch.empty((h, w), dtype=img.dtype, device=img.device)
    if out.dtype != img.dtype or tuple(out.shape) != (h, w) or out.stride(1) != 1:
        raise ValueError("out must match img")
    code = load().fx_hybrid_median(img.data_ptr(), w, h, img.stride(0) * img.element_size(), _dtype_code(img),
                                   int(window), out.data_ptr(), out.stride(0) * out.element_size(),
                                   _stream_ptr(stream))
    _check(code, "fx_hybrid_median")
    return out


def desc_for(img, out) -> ImageDesc:
    h, w = img.shape
    return ImageDesc(img.data_ptr(), w, h, img.stride(0) * img.element_size(), _dtype_code(img), 0,
                     out.data_ptr(), out.stride(0))


class Plan:
    """fx_plan: fixed parameters plus the batched path's device workspace."""

    def __init__(self, params: Params | None = None, max_images: int = 64, device: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        p = params if params is not None else make_params(FX_U16)
        _check(self._lib.fx_plan_create(ctypes.byref(self._h), ctypes.byref(p), max_images, device),
               "fx_plan_create")
        self.max_images = max_images

    def close(self):
        if self._h:
            _check(self._lib.fx_plan_destroy(self._h), "fx_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _descs(pairs):
        arr = (ImageDesc * len(pairs))()
        for i, (img, out) in enumerate(pairs):
            arr[i] = desc_for(img, out)
        return arr

    def extract_batch(self, pairs, stream=None):
        """pairs: list of (image tensor, output mask tensor)."""
        arr = self._descs(pairs)
        _check(self._lib.fx_extract_batch(self._h, arr, len(pairs), _stream_ptr(stream)), "fx_extract_batch")

    def autotune(self, pairs, stream=None):
        arr = self._descs(pairs)
        tw, th, cps = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.fx_plan_autotune(self._h, arr, len(pairs), _stream_ptr(stream), ctypes.byref(tw),
                                          ctypes.byref(th), ctypes.byref(cps)), "fx_plan_autotune")
        return tw.value, th.value, cps.value

    def set_tile(self, tile_w: int, tile_h: int, ctas_per_sm: int):
        _check(self._lib.fx_plan_set_tile(self._h, tile_w, tile_h, ctas_per_sm), "fx_plan_set_tile")

    def device_status(self, stream=None) -> int:
        return self._lib.fx_get_device_status(self._h, _stream_ptr(stream))

    def extract_host(self, img_np, out_np=None):
        """End to end on host numpy arrays (pinned memory copies fastest)."""
        import numpy as np
        if img_np.ndim != 2 or img_np.strides[1] != img_np.itemsize:
            raise ValueError("img must be 2-D with contiguous rows")
        h, w = img_np.shape
        dt = FX_U8 if img_np.dtype == np.uint8 else FX_U16 if img_np.dtype == np.uint16 else None
        if dt is None:
            raise TypeError(img_np.dtype)
        if out_np is None:
            out_np = np.empty((h, w), dtype=np.uint8)
        _check(self._lib.fx_extract_host(self._h, img_np.ctypes.data, w, h, img_np.strides[0], dt,
                                         out_np.ctypes.data, out_np.strides[0]), "fx_extract_host")
        return out_np

    def extract_host_batch(self, pairs):
        """fx_extract_host_batch on a list of (image, mask) host numpy arrays
        (2-D, contiguous rows); the masks are filled in place."""
        import numpy as np
        arr = (ImageDesc * len(pairs))()
        for i, (img, out) in enumerate(pairs):
            if img.ndim != 2 or img.strides[1] != img.itemsize or out.shape != img.shape or out.dtype != np.uint8:
                raise ValueError("pairs must be 2-D images with contiguous rows and uint8 masks of the same shape")
            dt = FX_U8 if img.dtype == np.uint8 else FX_U16 if img.dtype == np.uint16 else None
            if dt is None:
                raise TypeError(img.dtype)
            arr[i].img, arr[i].width, arr[i].height, arr[i].pitch_bytes = img.ctypes.data, img.shape[1], img.shape[0], img.strides[0]
            arr[i].dtype, arr[i].out_mask, arr[i].out_pitch = dt, out.ctypes.data, out.strides[0]
        _check(self._lib.fx_extract_host_batch(self._h, arr, len(pairs)), "fx_extract_host_batch")
        return [out for _, out in pairs]


def specialize(params: "Params", dtype: int) -> bool:
    """fx_specialize: compile the streaming first pass for these parameters
    and dtype (FX_U8 / FX_U16) on the current device; False when run-time
    compilation is unavailable (FX_ERR_UNSUPPORTED), an exception on other
    errors."""
    code = load().fx_specialize(ctypes.byref(params), dtype)
    if code == 2:
        return False
    _check(code, "fx_specialize")
    return True


def checked_violations(reset: bool = False):
    """Range-check failures counted by the checked build's kernels (None when
    the loaded library is the normal build)."""
    n = ctypes.c_uint64(0)
    code = load().fx_checked_violations(ctypes.byref(n), 1 if reset else 0)
    if code == 2:  # FX_ERR_UNSUPPORTED: not the checked build
        return None
    _check(code, "fx_checked_violations")
    return int(n.value)

