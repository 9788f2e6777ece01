"""CPU oracle for rectangular-element grayscale erosion/dilation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the GPU library and its Python binding never do, and the two share
no code.

The arithmetic lives in ``morph_oracle.c`` (plain C, OpenMP over rows); this
module only compiles it with gcc and marshals numpy arrays through ctypes.

Functions (all integer, so exact; see the C file's header for the citations):

* ``morph(src, wx, wy, ax, ay, op)`` -- the paper's section 2 definition by
  brute force over the clipped window (erosion: op='erode', min; dilation:
  op='dilate', max; pixels outside the image ignored).
* ``morph_points(src, wx, wy, ax, ay, op, xs, ys)`` -- the same definition at
  sample points only.
* ``sep_vhgw(src, wx, wy, ax, ay, op)`` -- separable van Herk/Gil-Werman
  checker (section 5, section 5.1.1).
* ``line_wedge(line, w, a, op)`` -- monotone-deque 1-D sliding min/max.
* ``transpose(src)`` -- section 4, D[j][i] = S[i][j].
* ``opening``, ``closing``, ``gradient`` -- section 2's compositions of
  erosion, dilation and arithmetic (the second step of an opening or closing
  by the reflected element; the gradient is dilation minus erosion by the
  same element).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "morph_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lib = None
_lock = threading.Lock()

_OPS = {"erode": 0, "dilate": 1, 0: 0, 1: 1}


def build(force: bool = False) -> str:
    """Compile ``morph_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        lib.oracle_morph.argtypes = [vp, i32, i32, i32, i64, i32, i32, i32, i32,
                                     i32, vp, i64]
        lib.oracle_morph_points.argtypes = [vp, i32, i32, i32, i64, i32, i32,
                                            i32, i32, i32, vp, vp, i64, vp]
        lib.oracle_sep_vhgw.argtypes = lib.oracle_morph.argtypes
        lib.oracle_line_wedge.argtypes = [vp, i64, i32, i32, i32, i32, vp]
        lib.oracle_transpose.argtypes = [vp, i32, i32, i32, i64, vp, i64]
        lib.oracle_num_threads.argtypes = []
        lib.oracle_set_threads.argtypes = [i32]
        for f in (lib.oracle_morph, lib.oracle_morph_points, lib.oracle_sep_vhgw,
                  lib.oracle_line_wedge, lib.oracle_transpose,
                  lib.oracle_num_threads, lib.oracle_set_threads):
            f.restype = ctypes.c_int
        _lib = lib
        return lib


def _image(src: np.ndarray) -> np.ndarray:
    if src.ndim != 2 or src.dtype not in (np.uint8, np.uint16):
        raise ValueError("oracle images are 2-D uint8 or uint16 arrays")
    return np.ascontiguousarray(src)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError("oracle %s rejected its arguments (rc=%d)" % (what, rc))


def morph(src: np.ndarray, wx: int, wy: int, ax: int | None = None,
          ay: int | None = None, op="erode") -> np.ndarray:
    """Brute-force erosion/dilation (section 2 definition)."""
    s = _image(src)
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    out = np.empty_like(s)
    h, w = s.shape
    rc = _load().oracle_morph(_ptr(s), s.itemsize, w, h, s.strides[0], wx, wy,
                              ax, ay, _OPS[op], _ptr(out), out.strides[0])
    _check(rc, "morph")
    return out


def morph_points(src: np.ndarray, wx: int, wy: int, ax: int | None, ay: int | None,
                 op, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """The section 2 definition evaluated at the points (xs[i], ys[i])."""
    s = _image(src)
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    if xs.shape != ys.shape or xs.ndim != 1:
        raise ValueError("xs and ys must be 1-D and of equal length")
    out = np.empty(xs.shape, dtype=np.uint32)
    h, w = s.shape
    rc = _load().oracle_morph_points(_ptr(s), s.itemsize, w, h, s.strides[0], wx,
                                     wy, ax, ay, _OPS[op], _ptr(xs), _ptr(ys),
                                     xs.size, _ptr(out))
    _check(rc, "morph_points")
    return out.astype(s.dtype)


def sep_vhgw(src: np.ndarray, wx: int, wy: int, ax: int | None = None,
             ay: int | None = None, op="erode") -> np.ndarray:
    """Separable van Herk/Gil-Werman checker (section 5, 5.1.1)."""
    s = _image(src)
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    out = np.empty_like(s)
    h, w = s.shape
    rc = _load().oracle_sep_vhgw(_ptr(s), s.itemsize, w, h, s.strides[0], wx, wy,
                                 ax, ay, _OPS[op], _ptr(out), out.strides[0])
    _check(rc, "sep_vhgw")
    return out


def line_wedge(line: np.ndarray, w: int, a: int, op="erode") -> np.ndarray:
    """Monotone-deque sliding min/max over a 1-D line (window start x-a)."""
    ln = np.ascontiguousarray(line, dtype=np.uint32)
    out = np.empty_like(ln)
    rc = _load().oracle_line_wedge(_ptr(ln), 1, ln.size, w, a, _OPS[op], _ptr(out))
    _check(rc, "line_wedge")
    return out


def wedge_separable(src: np.ndarray, wx: int, wy: int, ax: int | None = None,
                    ay: int | None = None, op="erode") -> np.ndarray:
    """Erosion/dilation as a deque pass along x, then one along y."""
    s = _image(src)
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    tmp = np.stack([line_wedge(row, wx, ax, op) for row in s.astype(np.uint32)])
    out = np.stack([line_wedge(col, wy, ay, op) for col in tmp.T]).T
    return out.astype(s.dtype)


def transpose(src: np.ndarray) -> np.ndarray:
    """Section 4 transpose, D[j][i] = S[i][j]."""
    s = _image(src)
    h, w = s.shape
    out = np.empty((w, h), dtype=s.dtype)
    rc = _load().oracle_transpose(_ptr(s), s.itemsize, w, h, s.strides[0],
                                  _ptr(out), out.strides[0])
    _check(rc, "transpose")
    return out


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> int:
    """Sets the OpenMP threads of later calls; returns the previous count."""
    return int(_load().oracle_set_threads(int(n)))


def reflect_anchor(w: int, a: int) -> int:
    """Anchor of the reflected element: the cell at offset a from the start
    of a window of length w sits at offset w-1-a once the window is mirrored."""
    return w - 1 - a


def opening(src: np.ndarray, wx: int, wy: int, ax: int | None = None,
            ay: int | None = None) -> np.ndarray:
    """Opening as erosion then dilation by the reflected element (section 2:
    other operations are compositions of erosion and dilation)."""
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    e = morph(src, wx, wy, ax, ay, "erode")
    return morph(e, wx, wy, reflect_anchor(wx, ax), reflect_anchor(wy, ay), "dilate")


def closing(src: np.ndarray, wx: int, wy: int, ax: int | None = None,
            ay: int | None = None) -> np.ndarray:
    """Closing as dilation then erosion by the reflected element."""
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    d = morph(src, wx, wy, ax, ay, "dilate")
    return morph(d, wx, wy, reflect_anchor(wx, ax), reflect_anchor(wy, ay), "erode")


def gradient(src: np.ndarray, wx: int, wy: int, ax: int | None = None,
             ay: int | None = None) -> np.ndarray:
    """Morphological gradient: dilation minus erosion by the same element and
    anchor (section 2: expressed through erosion, dilation and arithmetic).
    Never negative, so it fits the source's pixel type."""
    ax = wx // 2 if ax is None else ax
    ay = wy // 2 if ay is None else ay
    d = morph(src, wx, wy, ax, ay, "dilate")
    e = morph(src, wx, wy, ax, ay, "erode")
    return (d - e).astype(src.dtype)
