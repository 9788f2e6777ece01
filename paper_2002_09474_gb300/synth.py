"""Seeded synthetic inputs for the five workloads (host numpy, PCG64).

This module holds no erosion/dilation arithmetic: it only draws images and
request parameters.  Both the GPU-path tests/bench and the CPU oracle take
their inputs from here, so the two sides always see the same bytes.

The paper measures on a single 800x600 8-bit gray image (section 5.1.3,
5.2.3) and uses no public dataset; the generators below stand in for it at the
sizes of the five workloads:

* ``uniform_image``  -- i.i.d. uniform pixels (640x480 u8 seed 1; 4096^2 u8/u16)
* ``document_image`` -- 1920x1080 u8 "document": background 255, 300 dark
  rectangles and strokes with values 0..60 and sides 2..40, +-10 noise, clipped
* ``gradient_image`` -- 4096^2 smooth diagonal gradient plus uniform noise
* ``batch_specs``    -- 2000 images with sides uniform in 64..2048, windows
  uniform in 1..63, anchor floor(w/2), erode/dilate flag
* ``serving_requests`` -- Poisson arrivals, area log-uniform 128^2..4096^2,
  aspect log-uniform in [1/2, 2], windows uniform in 1..101, mixed ops
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ERODE = 0
DILATE = 1


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _maxval(dtype) -> int:
    return int(np.iinfo(dtype).max)


def uniform_image(width: int, height: int, dtype=np.uint8, seed: int = 1,
                  gen: np.random.Generator | None = None) -> np.ndarray:
    """i.i.d. uniform pixels over the full range of ``dtype``."""
    g = gen if gen is not None else rng(seed)
    return g.integers(0, _maxval(dtype), size=(height, width), dtype=dtype,
                      endpoint=True)


def gradient_image(width: int, height: int, dtype=np.uint8, seed: int = 3,
                   noise: int | None = None) -> np.ndarray:
    """floor(M*(x+y)/(W+H-2)) plus uniform noise in [-n, n], clipped to
    [0, M]; n defaults to 8 for 8-bit and 2048 for 16-bit pixels."""
    g = rng(seed)
    m = _maxval(dtype)
    if noise is None:
        noise = 8 if dtype == np.uint8 else 2048
    xs = np.arange(width, dtype=np.int64)[None, :]
    ys = np.arange(height, dtype=np.int64)[:, None]
    den = max(width + height - 2, 1)
    base = (m * (xs + ys)) // den
    nz = g.integers(-noise, noise, size=(height, width), endpoint=True,
                    dtype=np.int64)
    return np.clip(base + nz, 0, m).astype(dtype)


def document_image(width: int = 1920, height: int = 1080, seed: int = 2,
                   n_shapes: int = 300) -> np.ndarray:
    """Document-like page: background 255, ``n_shapes`` dark shapes (half
    filled rectangles with sides 2..40, half horizontal/vertical strokes of
    length 2..40 and thickness 2..4), values 0..60, then +-10 uniform noise,
    clipped to 0..255."""
    g = rng(seed)
    img = np.full((height, width), 255, dtype=np.int16)
    for i in range(n_shapes):
        val = int(g.integers(0, 60, endpoint=True))
        if i % 2 == 0:
            sw = int(g.integers(2, 40, endpoint=True))
            sh = int(g.integers(2, 40, endpoint=True))
        else:
            length = int(g.integers(2, 40, endpoint=True))
            thick = int(g.integers(2, 4, endpoint=True))
            if g.integers(0, 1, endpoint=True):
                sw, sh = length, thick
            else:
                sw, sh = thick, length
        x0 = int(g.integers(0, max(width - sw, 0), endpoint=True))
        y0 = int(g.integers(0, max(height - sh, 0), endpoint=True))
        img[y0:y0 + sh, x0:x0 + sw] = val
    img += g.integers(-10, 10, size=img.shape, endpoint=True, dtype=np.int16)
    return np.clip(img, 0, 255).astype(np.uint8)


@dataclass(frozen=True)
class ImageSpec:
    """One image of a batch: its size, window, anchor and operation."""
    width: int
    height: int
    wx: int
    wy: int
    ax: int
    ay: int
    op: int  # ERODE or DILATE


def batch_specs(n: int = 2000, seed: int = 5, side_lo: int = 64,
                side_hi: int = 2048, w_hi: int = 63) -> list[ImageSpec]:
    """Sizes, windows and ops of the batched workload: sides uniform in
    [side_lo, side_hi], windows uniform in 1..w_hi, anchor floor(w/2), op a
    fair coin."""
    g = rng(seed)
    ws = g.integers(side_lo, side_hi, size=n, endpoint=True)
    hs = g.integers(side_lo, side_hi, size=n, endpoint=True)
    wxs = g.integers(1, w_hi, size=n, endpoint=True)
    wys = g.integers(1, w_hi, size=n, endpoint=True)
    ops = g.integers(0, 1, size=n, endpoint=True)
    return [ImageSpec(int(ws[i]), int(hs[i]), int(wxs[i]), int(wys[i]),
                      int(wxs[i]) // 2, int(wys[i]) // 2, int(ops[i]))
            for i in range(n)]


def batch_pixels(specs: list[ImageSpec], seed: int = 5) -> list[np.ndarray]:
    """Uniform u8 pixels for every image of ``specs`` (a separate stream,
    so the specs do not depend on how many pixels are drawn)."""
    g = rng(seed + 1000)
    return [uniform_image(s.width, s.height, np.uint8, gen=g) for s in specs]


@dataclass(frozen=True)
class Request:
    """One filtering request of the serving workload."""
    arrival_s: float
    width: int
    height: int
    wx: int
    wy: int
    ax: int
    ay: int
    op: int


def serving_requests(rate_per_s: float, duration_s: float, seed: int = 6,
                     area_lo: int = 128 * 128, area_hi: int = 4096 * 4096,
                     w_hi: int = 101) -> list[Request]:
    """Poisson arrivals at ``rate_per_s`` for ``duration_s`` seconds; area
    log-uniform in [area_lo, area_hi], aspect ratio log-uniform in [1/2, 2],
    windows uniform in 1..w_hi, anchor floor(w/2), op a fair coin."""
    g = rng(seed)
    out: list[Request] = []
    t = 0.0
    while True:
        t += float(g.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        area = float(np.exp(g.uniform(np.log(area_lo), np.log(area_hi))))
        aspect = float(np.exp(g.uniform(np.log(0.5), np.log(2.0))))
        w = max(1, int(round(np.sqrt(area * aspect))))
        h = max(1, int(round(np.sqrt(area / aspect))))
        wx = int(g.integers(1, w_hi, endpoint=True))
        wy = int(g.integers(1, w_hi, endpoint=True))
        op = int(g.integers(0, 1, endpoint=True))
        out.append(Request(t, w, h, wx, wy, wx // 2, wy // 2, op))
    return out


# The five named workloads (window lists follow their descriptions).
C2_WINDOWS = (3, 7, 15, 31, 61)
C3_WINDOWS = ((1, 101), (101, 1), (21, 51), (127, 127))  # (wx, wy)
