"""GPU parity of the single-pass kernels against the CPU oracle, each forced
on in turn: the warp-tiled van Herk/Gil-Werman pass along y (section 5.1.1,
tile heights from 8 to 512 rows, strips 128 and 256 bytes wide), the register-blocked
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
    morph.morph_set_colv(-1, 0, 0)
    morph.morph_set_rowv(-1, 0)


def windows_1d(n):
    out = []
    for w in (2, 3, 8, 9, 16, 17, 31, 51, 64, 101, 127, 200, 255, 256, 300):
        for a in sorted({0, w // 2, w - 1}):
            out.append((w, a))
    return out


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("lanes", [4, 8])
@pytest.mark.parametrize("rows", [0, 8, 40, 128, 512])
def test_pass_along_y_warp_tiled(lib, dtype, lanes, rows):
    """lanes: bytes per lane -- 4 (strips 128 bytes wide), 8 (256 bytes, two
    words per lane)."""
    torch = need_cuda()
    g = synth.rng(300 + rows + lanes)
    try:
        assert lib.morph_set_colv(1, rows, lanes) == 0
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
        lib.morph_set_colv(-1, 0, 0)


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
        assert lib.morph_set_colv(0, 0, 0) == 0 and lib.morph_set_rowv(0, 0) == 0
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
        lib.morph_set_colv(-1, 0, 0)
        lib.morph_set_rowv(-1, 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_two_launch_form_with_new_passes(lib, dtype):
    """2-D windows as a pass along y into an intermediate and a pass along x
    from it, both by the new kernels, against the oracle."""
    torch = need_cuda()
    g = synth.rng(510)
    try:
        assert lib.morph_set_split(1) == 0
        assert lib.morph_set_colv(1, 0, 0) == 0 and lib.morph_set_rowv(1, 0) == 0
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
        lib.morph_set_colv(-1, 0, 0)
        lib.morph_set_rowv(-1, 0)
