"""The paper's CPU method on the host (sections 4 and 5): 8-bit erosion and
dilation as two separable passes with 16-lane NEON min/max and 16 x 16
block transposes on aarch64, and the same methods pixel by pixel as the
scalar baseline.

A CPU BASELINE for ``bench.py`` only (the paper's NEON-over-scalar ratios,
re-measured on the GPU machine's Arm host): the GPU library never imports it,
and the tests check it against the oracle.  The arithmetic lives in
``paper_cpu.c``; this module compiles it with gcc (without
auto-vectorisation, so the scalar form stays scalar) and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paper_cpu.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libpapercpu.so")

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``paper_cpu.c`` into ``cpu_method/_build/libpapercpu.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fno-tree-vectorize", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, lg, i32 = ctypes.c_void_p, ctypes.c_long, ctypes.c_int
            lib.cm_has_neon.argtypes = []
            lib.cm_morph_u8.argtypes = [vp, lg, vp, lg, i32, i32, i32, i32, i32, i32, i32, i32, i32]
            lib.cm_transpose_blocks.argtypes = [i32, i32, vp, vp, lg]
            for f in (lib.cm_has_neon, lib.cm_morph_u8, lib.cm_transpose_blocks):
                f.restype = i32
            _lib = lib
    return _lib


def has_neon() -> bool:
    """True where the NEON form is compiled in (aarch64 hosts)."""
    return bool(_load().cm_has_neon())


def morph(src: np.ndarray, wx: int, wy: int, ax: int | None = None, ay: int | None = None, op="erode",
          method: str = "direct", vector: bool = True) -> np.ndarray:
    """Erosion or dilation of a 2-D uint8 image (pixels outside the image
    ignored) by the paper's method: method 'direct' or 'vhgw' for both
    passes; vector True for the NEON form, False for the scalar one."""
    src = np.ascontiguousarray(src, dtype=np.uint8)
    h, w = src.shape
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    out = np.empty_like(src)
    rc = _load().cm_morph_u8(src.ctypes.data, w, out.ctypes.data, w, w, h, wx, wy, ax, ay,
                              0 if op in ("erode", 0) else 1, 1 if method == "vhgw" else 0, 1 if vector else 0)
    if rc != 0:
        raise RuntimeError("cm_morph_u8 failed (%d)" % rc)
    return out


def transpose_blocks(kind: str, blocks: np.ndarray, vector: bool = True) -> np.ndarray:
    """Transposes every block of ``blocks`` (kind 'u8': n x 16 x 16 uint8;
    'u16': n x 8 x 8 uint16)."""
    blocks = np.ascontiguousarray(blocks)
    out = np.empty_like(blocks)
    rc = _load().cm_transpose_blocks(0 if kind == "u8" else 1, 1 if vector else 0, blocks.ctypes.data,
                                     out.ctypes.data, blocks.shape[0])
    if rc != 0:
        raise RuntimeError("cm_transpose_blocks failed (%d)" % rc)
    return out
