"""GPU parity of the fused single-image path against the CPU oracle.

Bit-exact (integer min/max): every case compares all pixels with the
oracle's brute-force definition (section 2), with both pass methods forced in
turn (direct, section 5.1.2/5.2.2; van Herk/Gil-Werman, 5.1.1/5.2.1), every
tile shape, ragged image edges, pitched and unaligned buffers, and guard
bytes around the destination.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

from gpu_util import DeviceImage, need_cuda

pytestmark = pytest.mark.gpu

OPS = {"erode": 0, "dilate": 1}
DIRECT, VHGW = 10**6, 0  # crossover values that force one method on both passes


@pytest.fixture(scope="module")
def lib():
    need_cuda()
    from paper_2002_09474_gb300 import morph
    yield morph
    morph.morph_reset_tuning()


def aligned_pad(w, dtype):
    """Row padding that makes the pitch a multiple of 16 bytes (TMA path)."""
    row = w * np.dtype(dtype).itemsize
    return (16 - row % 16) % 16


def run(lib, torch, img, wx, wy, ax, ay, op, pad=0, offset=0, dst_pad=None, dst_offset=0):
    h, w = img.shape
    src = DeviceImage(torch, h, w, img.dtype, pad=pad, offset=offset, fill=img)
    dst = DeviceImage(torch, h, w, img.dtype, pad=pad if dst_pad is None else dst_pad,
                      offset=dst_offset)
    dtype = lib.MORPH_U8 if img.dtype == np.uint8 else lib.MORPH_U16
    rc = lib.morph_apply(src.ptr, src.pitch, dst.ptr, dst.pitch, w, h, dtype, OPS[op],
                         wx, wy, ax, ay, 0)
    assert rc == 0, lib.status_string(rc)
    torch.cuda.synchronize()
    assert lib.morph_device_error() == 0, "a kernel reported a device-side error"
    assert dst.untouched_outside(), "kernel wrote outside the destination image"
    assert src.untouched_outside()
    return dst.read()


def set_methods(lib, dtype, col, row, cfg=-1):
    code = lib.MORPH_U8 if dtype == np.uint8 else lib.MORPH_U16
    assert lib.morph_set_tuning(code, row, col, cfg) == 0


SHAPES = [(1, 1), (2, 3), (5, 17), (33, 7), (67, 130), (129, 257), (200, 300)]
WINDOWS = [(1, 1), (3, 3), (2, 5), (7, 1), (1, 9), (4, 4), (8, 8), (9, 16), (17, 8), (15, 15), (31, 7),
           (64, 65), (61, 61)]


@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("method", ["direct", "vhgw", "mixed"])
def test_shapes_windows_methods(lib, dtype, method, pipe):
    torch = need_cuda()
    lib.morph_reset_tuning()
    assert lib.morph_set_pipeline(pipe) == 0
    col, row = {"direct": (DIRECT, DIRECT), "vhgw": (VHGW, VHGW), "mixed": (DIRECT, VHGW)}[method]
    set_methods(lib, dtype, col, row)
    g = synth.rng(100 + (dtype == np.uint16))
    for (h, w) in SHAPES:
        img = synth.uniform_image(w, h, dtype, gen=g)
        for n, (wx, wy) in enumerate(WINDOWS):
            ax, ay = wx // 2, wy // 2
            for op in ("erode", "dilate"):
                # alternate plain-load (unaligned pitch) and TMA (aligned) paths
                pad = aligned_pad(w, dtype) if (n + (op == "dilate")) % 2 else 0
                got = run(lib, torch, img, wx, wy, ax, ay, op, pad=pad, dst_pad=pad)
                want = oracle.morph(img, wx, wy, ax, ay, op)
                assert np.array_equal(got, want), (h, w, wx, wy, op, method)


@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("cfg", [0, 1, 2, 3, 4, 5, 6, 7])
def test_every_tile_shape(lib, dtype, cfg, pipe):
    torch = need_cuda()
    lib.morph_reset_tuning()
    assert lib.morph_set_pipeline(pipe) == 0
    g = synth.rng(110 + cfg)
    img = synth.uniform_image(301, 177, dtype, gen=g)
    for method in ("direct", "vhgw"):
        c = DIRECT if method == "direct" else VHGW
        set_methods(lib, dtype, c, c, cfg)
        for (wx, wy, ax, ay) in ((3, 5, 1, 2), (8, 2, 7, 0), (21, 51, 10, 25), (101, 1, 50, 0),
                                 (1, 33, 0, 16), (127, 127, 63, 63)):
            for op in ("erode", "dilate"):
                for pad in (0, aligned_pad(301, dtype)):
                    got = run(lib, torch, img, wx, wy, ax, ay, op, pad=pad, dst_pad=pad)
                    want = oracle.morph(img, wx, wy, ax, ay, op)
                    assert np.array_equal(got, want), (cfg, method, wx, wy, op, pad)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_all_anchors_even_and_odd(lib, dtype):
    torch = need_cuda()
    lib.morph_reset_tuning()
    g = synth.rng(120)
    img = synth.uniform_image(70, 45, dtype, gen=g)
    for method in ("direct", "vhgw"):
        c = DIRECT if method == "direct" else VHGW
        set_methods(lib, dtype, c, c)
        for (wx, wy) in ((4, 3), (6, 6), (5, 2)):
            for ax, ay in itertools.product(range(wx), range(wy)):
                got = run(lib, torch, img, wx, wy, ax, ay, "erode")
                want = oracle.morph(img, wx, wy, ax, ay, "erode")
                assert np.array_equal(got, want), (method, wx, wy, ax, ay)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_pitched_and_unaligned_buffers(lib, dtype):
    """16-byte-aligned pitches take the TMA path; others the plain-load path;
    odd byte offsets force per-pixel loads and stores."""
    torch = need_cuda()
    lib.morph_reset_tuning()
    g = synth.rng(130)
    img = synth.uniform_image(150, 90, dtype, gen=g)
    esz = np.dtype(dtype).itemsize
    cases = [(0, 0, 0, 0), (16 - (150 * esz) % 16, 0, 32, 0), (13 * esz, 0, 13 * esz, 0),
             (6, 4, 2, 8), (esz, esz, 3 * esz, esz)]
    for pad, off, dpad, doff in cases:
        for (wx, wy) in ((3, 3), (17, 9), (40, 40)):
            for op in ("erode", "dilate"):
                got = run(lib, torch, img, wx, wy, wx // 2, wy // 2, op, pad=pad, offset=off,
                          dst_pad=dpad, dst_offset=doff)
                want = oracle.morph(img, wx, wy, wx // 2, wy // 2, op)
                assert np.array_equal(got, want), (pad, off, dpad, doff, wx, wy, op)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_windows_larger_than_image(lib, dtype):
    torch = need_cuda()
    lib.morph_reset_tuning()
    g = synth.rng(140)
    img = synth.uniform_image(37, 23, dtype, gen=g)
    for (wx, wy, ax, ay) in ((75, 47, 37, 23), (200, 3, 0, 1), (3, 500, 2, 499), (1000, 1000, 1, 998)):
        for op in ("erode", "dilate"):
            got = run(lib, torch, img, wx, wy, ax, ay, op)
            want = oracle.morph(img, wx, wy, ax, ay, op)
            assert np.array_equal(got, want), (wx, wy, ax, ay, op)


@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_tma_paths_on_whole_tiles(lib, dtype, pipe):
    """Sizes that are whole multiples of every tile shape with 16-byte
    pitches: every tile loads and stores through TMA."""
    torch = need_cuda()
    lib.morph_reset_tuning()
    assert lib.morph_set_pipeline(pipe) == 0
    g = synth.rng(150)
    img = synth.uniform_image(512, 256, dtype, gen=g)
    for cfg in range(8):
        for c in (DIRECT, VHGW):
            set_methods(lib, dtype, c, c, cfg)
            for (wx, wy) in ((3, 3), (1, 17), (17, 1), (21, 51)):
                for op in ("erode", "dilate"):
                    got = run(lib, torch, img, wx, wy, wx // 2, wy // 2, op)
                    want = oracle.morph(img, wx, wy, wx // 2, wy // 2, op)
                    assert np.array_equal(got, want), (cfg, c, wx, wy, op)


def test_constant_and_extreme_values(lib):
    torch = need_cuda()
    lib.morph_reset_tuning()
    for dtype in (np.uint8, np.uint16):
        mx = np.iinfo(dtype).max
        for v in (0, 1, mx - 1, mx):
            img = np.full((40, 50), v, dtype)
            for op in ("erode", "dilate"):
                assert np.array_equal(run(lib, torch, img, 5, 7, 2, 3, op), img)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_fused_and_two_launch_forms_agree(lib, dtype):
    """Section 5's separability through the two-launch form (1 x wy into an
    intermediate image, then wx x 1) and through the fused kernel."""
    torch = need_cuda()
    lib.morph_reset_tuning()
    g = synth.rng(160)
    try:
        for (h, w) in ((1, 1), (37, 300), (257, 129), (200, 513)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for (wx, wy, ax, ay) in ((2, 2, 0, 1), (9, 17, 4, 8), (127, 127, 63, 63), (40, 3, 39, 0)):
                want = {op: oracle.morph(img, wx, wy, ax, ay, op) for op in ("erode", "dilate")}
                for mode in (0, 1):
                    assert lib.morph_set_split(mode) == 0
                    for op in ("erode", "dilate"):
                        for pad in (0, aligned_pad(w, dtype)):
                            got = run(lib, torch, img, wx, wy, ax, ay, op, pad=pad, dst_pad=pad)
                            assert np.array_equal(got, want[op]), (h, w, wx, wy, mode, op, pad)
    finally:
        lib.morph_set_split(-1)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_persistent_form_many_tiles_per_cta(lib, dtype):
    """Images with several tiles per resident CTA, so each CTA of the
    persistent form uses both input slots many times; every tile shape,
    ragged right and bottom edges, against the separable checker and the
    one-CTA-per-tile form."""
    torch = need_cuda()
    g = synth.rng(170)
    h, w = 1900, 2501
    img = synth.uniform_image(w, h, dtype, gen=g)
    pad = aligned_pad(w, dtype)
    wins = ((3, 3), (1, 101), (101, 1), (21, 51), (127, 127), (9, 16))
    want = {(wx, wy, op): oracle.sep_vhgw(img, wx, wy, wx // 2, wy // 2, op)
            for (wx, wy) in wins for op in ("erode", "dilate")}
    try:
        for cfg in range(8):
            for (wx, wy) in wins:
                lib.morph_reset_tuning()
                set_methods(lib, dtype, 9, 9, cfg)
                for op in ("erode", "dilate"):
                    for pipe in (1, 0):
                        assert lib.morph_set_pipeline(pipe) == 0
                        assert lib.morph_set_split(0) == 0
                        got = run(lib, torch, img, wx, wy, wx // 2, wy // 2, op, pad=pad, dst_pad=pad)
                        assert np.array_equal(got, want[(wx, wy, op)]), (cfg, wx, wy, op, pipe)
    finally:
        lib.morph_reset_tuning()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_pass_along_x_through_transpose_kernels(lib, dtype):
    """Section 5.2.1's baseline form of the pass along x (transpose kernels,
    pass along y, transpose back) gives the same result as the fused form."""
    torch = need_cuda()
    lib.morph_reset_tuning()
    code = lib.MORPH_U8 if dtype == np.uint8 else lib.MORPH_U16
    g = synth.rng(180)
    try:
        for (h, w) in ((1, 1), (37, 300), (257, 129), (200, 513), (64, 64)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for (wx, wy, ax, ay) in ((5, 1, 2, 0), (64, 1, 10, 0), (127, 1, 63, 0), (9, 17, 4, 8),
                                     (40, 3, 39, 0), (2, 2, 1, 0)):
                for op in ("erode", "dilate"):
                    want = oracle.morph(img, wx, wy, ax, ay, op)
                    for mode in (1, 0):
                        assert lib.morph_set_xpass(code, mode) == 0
                        for pad in (0, aligned_pad(w, dtype)):
                            got = run(lib, torch, img, wx, wy, ax, ay, op, pad=pad, dst_pad=pad)
                            assert np.array_equal(got, want), (h, w, wx, wy, ax, ay, op, mode, pad)
    finally:
        lib.morph_reset_tuning()
