"""GPU parity of the single-pass kernels against the CPU oracle, each forced
on in turn: the warp-tiled van Herk/Gil-Werman pass along y (section 5.1.1,
tile heights from 8 to 512 rows) and its shared-tile form, the register-blocked
pass along x (sections 4 and 5.1.1's decomposition on 8-pixel blocks, every
segment length), and the older column and row kernels.  Bit-exact over ragged
shapes, anchor extremes, even and odd windows, pitched and unaligned buffers,
with guard bytes around the destination."""
import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

from gpu_util import need_cuda
from test_gpu_fused import aligned_pad, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    need_cuda()
    from paper_2002_09474_gb300 import morph
    yield morph
    morph.morph_reset_tuning()
    morph.morph_set_colv(-1, 0)
    morph.morph_set_rowv(-1, 0)


def windows_1d(n):
    out = []
    for w in (2, 3, 8, 9, 16, 17, 31, 51, 64, 101, 127, 200, 255, 256, 300):
        for a in sorted({0, w // 2, w - 1}):
            out.append((w, a))
    return out


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("mode", [1, 4, 6])
@pytest.mark.parametrize("rows", [0, 8, 40, 128, 512])
def test_pass_along_y_warp_tiled(lib, dtype, mode, rows):
    """mode 1: one word per lane (128-byte strips); 4: two (256-byte); 6:
    the ring form where rows are TMA-loadable (the tile's rows cycle
    through a few boxes), the whole-tile form elsewhere."""
    torch = need_cuda()
    g = synth.rng(300 + rows + mode)
    try:
        assert lib.morph_set_colv(mode, rows) == 0
        for (h, w) in ((1, 64), (37, 300), (300, 37), (1000, 129), (129, 1000), (2049, 64)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for i, (wy, ay) in enumerate(windows_1d(h)):
                if i % 3 != (h + w) % 3:
                    continue
                op = ("erode", "dilate")[i % 2]
                want = oracle.morph(img, 1, wy, 0, ay, op)
                pad = aligned_pad(w, dtype) if i % 2 else 3 * np.dtype(dtype).itemsize
                off = 0 if i % 4 < 2 else np.dtype(dtype).itemsize
                got = run(lib, torch, img, 1, wy, 0, ay, op, pad=pad, offset=off, dst_pad=pad)
                assert np.array_equal(got, want), (h, w, wy, ay, op, pad, off, rows)
    finally:
        lib.morph_set_colv(-1, 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("rows", [0, 8, 64, 300])
def test_pass_along_y_strip_streaming(lib, dtype, rows):
    """The strip-streaming form (8-row blocks, the rows w - 1 behind read a
    second time) for 9 <= wy <= 256 and TMA-loadable rows; band heights
    forced or planned; windows outside that range fall back to the warp
    tiles."""
    torch = need_cuda()
    g = synth.rng(340 + rows)
    esz = np.dtype(dtype).itemsize
    try:
        assert lib.morph_set_colv(5, rows) == 0
        for (h, w) in ((16, 128), (17, 640), (40, 300), (300, 129), (1000, 257), (2049, 64)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for i, (wy, ay) in enumerate(((9, 4), (10, 0), (16, 15), (17, 8), (33, 0), (64, 63), (65, 32),
                                          (101, 50), (127, 0), (256, 255), (5, 2), (300, 150))):
                op = ("erode", "dilate")[(i + h) % 2]
                want = oracle.morph(img, 1, wy, 0, ay, op)
                pad = aligned_pad(w, dtype)
                dpad, doff = (pad, 0) if i % 2 else (esz, 3 * esz)
                got = run(lib, torch, img, 1, wy, 0, ay, op, pad=pad, dst_pad=dpad, dst_offset=doff)
                assert np.array_equal(got, want), (h, w, wy, ay, op, rows)
    finally:
        lib.morph_set_colv(-1, 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_pass_along_y_shared_tile(lib, dtype):
    """The shared-tile form (warps share one input tile, block suffix in
    registers) for windows longer than 32 rows, TMA-loadable rows."""
    torch = need_cuda()
    g = synth.rng(350)
    try:
        assert lib.morph_set_colv(2, 0) == 0
        for (h, w) in ((40, 300), (300, 129), (1000, 257), (2049, 64)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for i, (wy, ay) in enumerate(((33, 0), (40, 39), (63, 31), (64, 0), (65, 64), (101, 50),
                                          (127, 0), (255, 127), (300, 299))):
                op = ("erode", "dilate")[i % 2]
                want = oracle.morph(img, 1, wy, 0, ay, op)
                pad = aligned_pad(w, dtype)
                dpad, doff = (pad, 0) if i % 2 else (np.dtype(dtype).itemsize, 3 * np.dtype(dtype).itemsize)
                got = run(lib, torch, img, 1, wy, 0, ay, op, pad=pad, dst_pad=dpad, dst_offset=doff)
                assert np.array_equal(got, want), (h, w, wy, ay, op)
    finally:
        lib.morph_set_colv(-1, 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("rows", [2, 3, 4])
@pytest.mark.parametrize("seg", [0, 256, 512, 2048])
def test_pass_along_x_register_blocked(lib, dtype, rows, seg):
    """rows: mode 2, 3 or 4 (8, 4 or 2 rows per warp)."""
    torch = need_cuda()
    g = synth.rng(400 + seg + rows)
    try:
        assert lib.morph_set_rowv(rows, seg) == 0
        for (h, w) in ((1, 64), (37, 300), (300, 37), (64, 1000), (13, 2049), (70, 257)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for i, (wx, ax) in enumerate(windows_1d(w)):
                if i % 3 != (h + w) % 3:
                    continue
                op = ("erode", "dilate")[i % 2]
                want = oracle.morph(img, wx, 1, ax, 0, op)
                pad = aligned_pad(w, dtype)
                dpad, doff = (pad, 0) if i % 2 else (np.dtype(dtype).itemsize, 3 * np.dtype(dtype).itemsize)
                got = run(lib, torch, img, wx, 1, ax, 0, op, pad=pad, dst_pad=dpad, dst_offset=doff)
                assert np.array_equal(got, want), (h, w, wx, ax, op, seg, dpad, doff)
    finally:
        lib.morph_set_rowv(-1, 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_older_single_pass_kernels(lib, dtype):
    """The column and row kernels that the new ones replace by default still
    give the oracle's result."""
    torch = need_cuda()
    g = synth.rng(500)
    try:
        assert lib.morph_set_colv(0, 0) == 0 and lib.morph_set_rowv(0, 0) == 0
        for (h, w) in ((37, 300), (300, 37), (257, 513)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for (wx, wy, ax, ay) in ((1, 101, 0, 50), (101, 1, 50, 0), (1, 9, 0, 8), (17, 1, 0, 0),
                                     (21, 51, 10, 25), (127, 127, 63, 63)):
                for op in ("erode", "dilate"):
                    want = oracle.morph(img, wx, wy, ax, ay, op)
                    pad = aligned_pad(w, dtype)
                    got = run(lib, torch, img, wx, wy, ax, ay, op, pad=pad, dst_pad=pad)
                    assert np.array_equal(got, want), (h, w, wx, wy, op)
    finally:
        lib.morph_set_colv(-1, 0)
        lib.morph_set_rowv(-1, 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_two_launch_form_with_new_passes(lib, dtype):
    """2-D windows as a pass along y into an intermediate and a pass along x
    from it, both by the new kernels, against the oracle."""
    torch = need_cuda()
    g = synth.rng(510)
    try:
        assert lib.morph_set_split(1) == 0
        assert lib.morph_set_colv(1, 0) == 0 and lib.morph_set_rowv(1, 0) == 0
        for (h, w) in ((37, 300), (300, 37), (511, 1025)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for (wx, wy, ax, ay) in ((21, 51, 10, 25), (127, 127, 63, 63), (9, 2, 0, 1), (256, 40, 255, 0)):
                for op in ("erode", "dilate"):
                    want = oracle.morph(img, wx, wy, ax, ay, op)
                    pad = aligned_pad(w, dtype)
                    for order in (0, 1):
                        assert lib.morph_set_split_order(order) == 0
                        got = run(lib, torch, img, wx, wy, ax, ay, op, pad=pad, dst_pad=pad)
                        assert np.array_equal(got, want), (h, w, wx, wy, op, order)
    finally:
        lib.morph_set_split(-1)
        lib.morph_set_split_order(1)
        lib.morph_set_colv(-1, 0)
        lib.morph_set_rowv(-1, 0)
