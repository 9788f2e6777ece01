"""Python binding of the C ABI in include/morph.h and include/morph_tuning.h
(ctypes).

Argument marshalling only: every function forwards to the entry point of the
same name in libmorph.so, and every pixel is computed by that library's CUDA
kernels.  There is no Python or CPU fallback: importing this module without
the built library raises.

Device pointers are plain integers (``tensor.data_ptr()``), streams are
``cudaStream_t`` values as integers (``torch.cuda.current_stream().cuda_stream``)
or 0 for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmorph.so")
HEADERS = [os.path.join(os.path.dirname(_PKG), "include", h) for h in ("morph.h", "morph_tuning.h")]

MORPH_OK = 0
MORPH_U8, MORPH_U16 = 0, 1
MORPH_ERODE, MORPH_DILATE = 0, 1
MORPH_OPEN, MORPH_CLOSE, MORPH_GRADIENT = 0, 1, 2
MORPH_NOALLOC_MAX_IMAGES = 256


class MorphError(RuntimeError):
    """A negative morph_status returned by the library."""

    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (fn, status_string(status), status))


class MorphDesc(ctypes.Structure):
    """morph_desc of include/morph.h (one image of a batch)."""
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("src_pitch", ctypes.c_int64), ("dst_pitch", ctypes.c_int64),
                ("wx", ctypes.c_int16), ("wy", ctypes.c_int16),
                ("anchor_x", ctypes.c_int16), ("anchor_y", ctypes.c_int16),
                ("op", ctypes.c_uint8), ("dtype", ctypes.c_uint8),
                ("pad", ctypes.c_uint8 * 2)]


class MorphCopyDesc(ctypes.Structure):
    """morph_copy_desc of include/morph.h (one contiguous copy)."""
    _fields_ = [("dst", ctypes.c_void_p), ("src", ctypes.c_void_p), ("bytes", ctypes.c_uint64)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libmorph.so is not built (%s); run paper_2002_09474_gb300.build.build() "
            "-- there is no CPU fallback" % LIB_PATH)
    return ctypes.CDLL(LIB_PATH)


_lib = _load()

_vp, _i32, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
_SIGS = {
    "morph_erode": [_vp, _i32, _i32, _sz, _i32, _i32, _i32, _i32, _vp, _vp],
    "morph_dilate": [_vp, _i32, _i32, _sz, _i32, _i32, _i32, _i32, _vp, _vp],
    "morph_erode_u16": [_vp, _i32, _i32, _sz, _i32, _i32, _i32, _i32, _vp, _vp],
    "morph_dilate_u16": [_vp, _i32, _i32, _sz, _i32, _i32, _i32, _i32, _vp, _vp],
    "morph_apply": [_vp, _sz, _vp, _sz, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _vp],
    "morph_composite": [_vp, _sz, _vp, _sz, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _vp],
    "morph_copy_2d": [_vp, _sz, _vp, _sz, _sz, _i32, _vp],
    "morph_copy_batch": [ctypes.POINTER(MorphCopyDesc), _i32, _vp],
    "morph_selftest_wait_timeout": [_vp],
    "morph_apply_host": [_vp, _sz, _vp, _sz, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _vp],
    "morph_release_staging": [],
    "morph_apply_host_batch": [ctypes.POINTER(MorphDesc), _i32, _vp],
    "morph_batch": [ctypes.POINTER(MorphDesc), _i32, _vp],
    "morph_batch_noalloc": [ctypes.POINTER(MorphDesc), _i32, _vp],
    "morph_batch_plan_create": [ctypes.POINTER(MorphDesc), _i32, ctypes.POINTER(_vp)],
    "morph_batch_plan_launch": [_vp, _vp],
    "morph_batch_plan_destroy": [_vp],
    "transpose_u8": [_vp, _i32, _i32, _sz, _vp, _sz, _vp],
    "transpose_u16": [_vp, _i32, _i32, _sz, _vp, _sz, _vp],
    "morph_autotune": [ctypes.c_char_p],
    "morph_status_string": [_i32],
    "morph_set_tuning": [_i32, _i32, _i32, _i32],
    "morph_reset_tuning": [],
    "morph_set_split": [_i32],
    "morph_set_split_order": [_i32],
    "morph_set_pdl": [_i32],
    "morph_set_pipeline": [_i32],
    "morph_set_column_kernel": [_i32],
    "morph_set_row_kernel": [_i32],
    "morph_set_colv": [_i32, _i32, _i32],
    "morph_set_rowv": [_i32, _i32],
    "morph_set_xpass": [_i32, _i32],
    "morph_set_batch_alone": [ctypes.c_longlong],
    "morph_set_composite_kernel": [_i32],
    "morph_device_error": [],
    "morph_launch_count": [],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name, None)
    if _f is None:
        continue
    _f.argtypes = _args
    _f.restype = (ctypes.c_char_p if _name == "morph_status_string" else
                  ctypes.c_longlong if _name == "morph_launch_count" else ctypes.c_int)


def declared_functions() -> list[str]:
    """Names of the functions the headers in include/ declare."""
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:long\s+long|[a-z_0-9]+)\s*\*?\s*([a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


def exported(name: str) -> bool:
    return getattr(_lib, name, None) is not None


def status_string(status: int) -> str:
    return _lib.morph_status_string(int(status)).decode()


def _check(fn: str, rc: int) -> int:
    if rc != MORPH_OK:
        raise MorphError(fn, rc)
    return rc


# ---- the C entry points, same names and arguments ----------------------------

def morph_erode(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream=0):
    return _lib.morph_erode(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream)


def morph_dilate(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream=0):
    return _lib.morph_dilate(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream)


def morph_erode_u16(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream=0):
    return _lib.morph_erode_u16(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream)


def morph_dilate_u16(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream=0):
    return _lib.morph_dilate_u16(src, width, height, pitch, wx, wy, anchor_x, anchor_y, dst, stream)


def morph_apply(src, src_pitch, dst, dst_pitch, width, height, dtype, op, wx, wy,
                anchor_x, anchor_y, stream=0):
    return _lib.morph_apply(src, src_pitch, dst, dst_pitch, width, height, dtype, op, wx, wy,
                            anchor_x, anchor_y, stream)


def morph_composite(src, src_pitch, dst, dst_pitch, width, height, dtype, kind, wx, wy,
                    anchor_x, anchor_y, stream=0):
    return _lib.morph_composite(src, src_pitch, dst, dst_pitch, width, height, dtype, kind, wx, wy,
                                anchor_x, anchor_y, stream)


def morph_selftest_wait_timeout(stream=0):
    return _lib.morph_selftest_wait_timeout(stream)


def morph_copy_2d(dst, dst_pitch, src, src_pitch, width_bytes, height, stream=0):
    return _lib.morph_copy_2d(dst, dst_pitch, src, src_pitch, width_bytes, height, stream)


def morph_copy_batch(copies, n, stream=0):
    return _lib.morph_copy_batch(copies, n, stream)


def morph_apply_host(src, src_pitch, dst, dst_pitch, width, height, dtype, op, wx, wy,
                     anchor_x, anchor_y, stream=0):
    return _lib.morph_apply_host(src, src_pitch, dst, dst_pitch, width, height, dtype, op, wx,
                                 wy, anchor_x, anchor_y, stream)


def morph_release_staging():
    return _lib.morph_release_staging()


def morph_apply_host_batch(descs, n, stream=0):
    return _lib.morph_apply_host_batch(descs, n, stream)


def morph_batch(descs, n, stream=0):
    return _lib.morph_batch(descs, n, stream)


def morph_batch_noalloc(descs, n, stream=0):
    return _lib.morph_batch_noalloc(descs, n, stream)


def morph_batch_plan_create(descs, n, plan_out):
    return _lib.morph_batch_plan_create(descs, n, plan_out)


def morph_batch_plan_launch(plan, stream=0):
    return _lib.morph_batch_plan_launch(plan, stream)


def morph_batch_plan_destroy(plan):
    return _lib.morph_batch_plan_destroy(plan)


def transpose_u8(src, width, height, src_pitch, dst, dst_pitch, stream=0):
    return _lib.transpose_u8(src, width, height, src_pitch, dst, dst_pitch, stream)


def transpose_u16(src, width, height, src_pitch, dst, dst_pitch, stream=0):
    return _lib.transpose_u16(src, width, height, src_pitch, dst, dst_pitch, stream)


def morph_autotune(cache_path=None):
    return _lib.morph_autotune(None if cache_path is None else str(cache_path).encode())


def morph_set_tuning(dtype, cross_row, cross_col, tile_cfg):
    return _lib.morph_set_tuning(dtype, cross_row, cross_col, tile_cfg)


def morph_set_split(mode):
    return _lib.morph_set_split(mode)


def morph_set_split_order(order):
    return _lib.morph_set_split_order(order)


def morph_set_pdl(on):
    return _lib.morph_set_pdl(on)


def morph_set_pipeline(mode):
    return _lib.morph_set_pipeline(mode)


def morph_set_column_kernel(mode):
    return _lib.morph_set_column_kernel(mode)


def morph_set_row_kernel(mode):
    return _lib.morph_set_row_kernel(mode)


def morph_set_colv(mode, rows=0, lane_bytes=0):
    return _lib.morph_set_colv(mode, rows, lane_bytes)


def morph_launch_count():
    return _lib.morph_launch_count()


def morph_set_rowv(mode, seg=0):
    return _lib.morph_set_rowv(mode, seg)


def morph_set_xpass(dtype, mode):
    return _lib.morph_set_xpass(dtype, mode)


def morph_set_batch_alone(min_pixels):
    return _lib.morph_set_batch_alone(min_pixels)


def morph_set_composite_kernel(mode):
    return _lib.morph_set_composite_kernel(mode)


def morph_reset_tuning():
    return _lib.morph_reset_tuning()


def morph_status_string(status):
    return _lib.morph_status_string(status)


def morph_device_error():
    return _lib.morph_device_error()


# ---- torch conveniences (marshalling only) -------------------------------------

def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.uint8:
        return MORPH_U8
    if t.dtype == torch.uint16:
        return MORPH_U16
    raise TypeError("images must be torch.uint8 or torch.uint16, got %s" % t.dtype)


def _pitch(t) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("images must be 2-D with unit stride along x")
    return t.stride(0) * t.element_size()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream))


def apply(src, dst, wx: int, wy: int, anchor_x: int | None = None, anchor_y: int | None = None,
          op: int = MORPH_ERODE, stream=None) -> None:
    """morph_apply on two CUDA tensors of shape (height, width) (rows may be
    strided).  Raises MorphError on a negative status."""
    if src.shape != dst.shape or src.dtype != dst.dtype:
        raise ValueError("src and dst must have the same shape and dtype")
    if not (src.is_cuda and dst.is_cuda):
        raise ValueError("src and dst must be CUDA tensors (use apply_host for host images)")
    h, w = src.shape
    ax = wx // 2 if anchor_x is None else anchor_x
    ay = wy // 2 if anchor_y is None else anchor_y
    _check("morph_apply", morph_apply(src.data_ptr(), _pitch(src), dst.data_ptr(), _pitch(dst),
                                      w, h, _dtype_code(src), op, wx, wy, ax, ay,
                                      _stream_handle(stream)))


def composite(src, dst, kind: int, wx: int, wy: int, anchor_x: int | None = None,
              anchor_y: int | None = None, stream=None) -> None:
    """morph_composite (MORPH_OPEN, MORPH_CLOSE or MORPH_GRADIENT) on two
    CUDA tensors of shape (height, width).  Raises MorphError on a negative
    status."""
    if src.shape != dst.shape or src.dtype != dst.dtype:
        raise ValueError("src and dst must have the same shape and dtype")
    if not (src.is_cuda and dst.is_cuda):
        raise ValueError("src and dst must be CUDA tensors")
    h, w = src.shape
    ax = wx // 2 if anchor_x is None else anchor_x
    ay = wy // 2 if anchor_y is None else anchor_y
    _check("morph_composite", morph_composite(src.data_ptr(), _pitch(src), dst.data_ptr(), _pitch(dst),
                                              w, h, _dtype_code(src), kind, wx, wy, ax, ay,
                                              _stream_handle(stream)))


def apply_host(src, dst, wx: int, wy: int, anchor_x: int | None = None, anchor_y: int | None = None,
               op: int = MORPH_ERODE, stream=None) -> None:
    """morph_apply_host on two host tensors (pinned for full copy speed)."""
    if src.shape != dst.shape or src.dtype != dst.dtype:
        raise ValueError("src and dst must have the same shape and dtype")
    h, w = src.shape
    ax = wx // 2 if anchor_x is None else anchor_x
    ay = wy // 2 if anchor_y is None else anchor_y
    _check("morph_apply_host", morph_apply_host(src.data_ptr(), _pitch(src), dst.data_ptr(),
                                                _pitch(dst), w, h, _dtype_code(src), op, wx, wy,
                                                ax, ay, _stream_handle(stream)))


def transpose(src, dst, stream=None) -> None:
    """transpose_u8/u16 of a (height, width) CUDA tensor into (width, height)."""
    h, w = src.shape
    if tuple(dst.shape) != (w, h) or dst.dtype != src.dtype:
        raise ValueError("dst must be (width, height) with the source dtype")
    fn = transpose_u8 if _dtype_code(src) == MORPH_U8 else transpose_u16
    _check(fn.__name__, fn(src.data_ptr(), w, h, _pitch(src), dst.data_ptr(), _pitch(dst),
                           _stream_handle(stream)))


def check_device_error() -> None:
    """Raises if a kernel reported a bounded-wait timeout (synchronises)."""
    v = morph_device_error()
    if v != 0:
        raise MorphError("device", -11 if v > 0 else v)
