"""GPU parity of the composite operations (section 2: opening, closing and
the morphological gradient through erosion, dilation and arithmetic) called
as one library call, bit-exact against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

from gpu_util import DeviceImage, need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    need_cuda()
    from paper_2002_09474_gb300 import morph
    morph.morph_reset_tuning()
    yield morph


def want_of(kind, img, wx, wy, ax, ay, lib):
    if kind == lib.MORPH_OPEN:
        return oracle.opening(img, wx, wy, ax, ay)
    if kind == lib.MORPH_CLOSE:
        return oracle.closing(img, wx, wy, ax, ay)
    return oracle.gradient(img, wx, wy, ax, ay)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_composite_shapes_windows_anchors_pitches(lib, dtype):
    torch = need_cuda()
    g = synth.rng(950)
    esz = np.dtype(dtype).itemsize
    code = lib.MORPH_U8 if dtype == np.uint8 else lib.MORPH_U16
    kinds = (lib.MORPH_OPEN, lib.MORPH_CLOSE, lib.MORPH_GRADIENT)
    n = 0
    for (h, w) in ((1, 1), (5, 3), (37, 300), (300, 129), (700, 257)):
        img = synth.uniform_image(w, h, dtype, gen=g)
        for (wx, wy, ax, ay) in ((1, 1, 0, 0), (3, 3, 1, 1), (4, 6, 0, 5), (21, 51, 10, 25), (101, 1, 50, 0),
                                 (1, 101, 0, 100), (127, 127, 63, 63), (9, 16, 8, 0)):
            for kind in kinds:
                n += 1
                spad = (16 - (w * esz) % 16) % 16 if n % 2 else 3 * esz
                src = DeviceImage(torch, h, w, dtype, pad=spad, offset=esz * (n % 3 == 0), fill=img)
                dst = DeviceImage(torch, h, w, dtype, pad=esz * (n % 4))
                rc = lib.morph_composite(src.ptr, src.pitch, dst.ptr, dst.pitch, w, h, code, kind, wx, wy, ax, ay, 0)
                assert rc == 0, lib.status_string(rc)
                torch.cuda.synchronize()
                assert dst.untouched_outside()
                np.testing.assert_array_equal(dst.read(), want_of(kind, img, wx, wy, ax, ay, lib),
                                              err_msg=str((h, w, wx, wy, ax, ay, kind)))
    assert lib.morph_device_error() == 0


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_composite_large_against_separable_checker(lib, dtype):
    """A 2048 x 1536 image with long windows (the single-pass kernels and the
    two-launch form inside each step), against the separable checker, which
    is pinned to the brute force by the CPU tests; and the three kinds'
    algebra: opening <= image <= closing, gradient = dilate - erode."""
    torch = need_cuda()
    img = synth.gradient_image(2048, 1536, dtype, seed=951)
    s = torch.from_numpy(img).cuda()
    wx, wy, ax, ay = 31, 101, 15, 50
    rx, ry = wx - 1 - ax, wy - 1 - ay
    ero = oracle.sep_vhgw(img, wx, wy, ax, ay, "erode")
    dil = oracle.sep_vhgw(img, wx, wy, ax, ay, "dilate")
    want = {lib.MORPH_OPEN: oracle.sep_vhgw(ero, wx, wy, rx, ry, "dilate"),
            lib.MORPH_CLOSE: oracle.sep_vhgw(dil, wx, wy, rx, ry, "erode"),
            lib.MORPH_GRADIENT: (dil - ero).astype(dtype)}
    for kind, w_ in want.items():
        o = torch.empty_like(s)
        lib.composite(s, o, kind, wx, wy, ax, ay)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o.cpu().numpy(), w_, err_msg=str(kind))
    assert (want[lib.MORPH_OPEN] <= img).all() and (img <= want[lib.MORPH_CLOSE]).all()


def test_composite_in_a_cuda_graph_and_errors(lib):
    """The call captures into a CUDA graph (its scratch is stream-ordered)
    and replays exactly; bad kinds, windows and aliasing are rejected."""
    torch = need_cuda()
    img = synth.uniform_image(640, 480, np.uint8, seed=952)
    s = torch.from_numpy(img).cuda()
    o = torch.empty_like(s)
    want = oracle.gradient(img, 7, 5, 3, 2)
    lib.composite(s, o, lib.MORPH_GRADIENT, 7, 5, 3, 2)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lib.composite(s, o, lib.MORPH_GRADIENT, 7, 5, 3, 2, stream=torch.cuda.current_stream())
    for _ in range(3):
        o.zero_()
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o.cpu().numpy(), want)
    p = s.data_ptr()
    assert lib.morph_composite(p, 640, o.data_ptr(), 640, 640, 480, lib.MORPH_U8, 3, 3, 3, 1, 1, 0) == -10
    assert lib.morph_composite(p, 640, o.data_ptr(), 640, 640, 480, lib.MORPH_U8, 0, 0, 3, 0, 1, 0) == -3
    assert lib.morph_composite(p, 640, p, 640, 640, 480, lib.MORPH_U8, 1, 3, 3, 1, 1, 0) == -6
    lib.check_device_error()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_one_pass_composite_small_windows(lib, dtype):
    """Windows of at most 9 x 9 through the one-pass kernel (forced for every
    kind): one launch per call, every pixel equal to the oracle's composite
    and to the two-call form's, over ragged sizes (tile edges inside and
    beyond the image), anchor extremes, offsets and unaligned pitches; by
    default the gradient of windows up to 5 x 5 takes it."""
    torch = need_cuda()
    g = synth.rng(952)
    esz = np.dtype(dtype).itemsize
    code = lib.MORPH_U8 if dtype == np.uint8 else lib.MORPH_U16
    kinds = (lib.MORPH_OPEN, lib.MORPH_CLOSE, lib.MORPH_GRADIENT)
    n = 0
    try:
        for (h, w) in ((9, 9), (33, 129), (95, 300), (1500, 700)):
            img = synth.uniform_image(w, h, dtype, gen=g)
            for (wx, wy) in ((1, 9), (9, 1), (2, 2), (3, 5), (8, 9), (9, 9)):
                for kind in kinds:
                    n += 1
                    ax, ay = (0, wx // 2, wx - 1)[n % 3], (wy - 1, 0, wy // 2)[n % 3]
                    spad = (16 - (w * esz) % 16) % 16 if n % 2 else 3 * esz
                    src = DeviceImage(torch, h, w, dtype, pad=spad, offset=esz * (n % 3 == 0), fill=img)
                    outs = []
                    for mode in (1, 0):
                        assert lib.morph_set_composite_kernel(mode) == 0
                        dst = DeviceImage(torch, h, w, dtype, pad=esz * (n % 4))
                        torch.cuda.synchronize()
                        n0 = lib.morph_launch_count()
                        rc = lib.morph_composite(src.ptr, src.pitch, dst.ptr, dst.pitch, w, h, code, kind, wx, wy,
                                                 ax, ay, 0)
                        assert rc == 0, lib.status_string(rc)
                        torch.cuda.synchronize()
                        if mode == 1:
                            assert lib.morph_launch_count() - n0 == 1, "not the one-pass kernel"
                        assert dst.untouched_outside()
                        outs.append(dst.read())
                    want = want_of(kind, img, wx, wy, ax, ay, lib)
                    err = str((h, w, wx, wy, ax, ay, kind))
                    np.testing.assert_array_equal(outs[0], want, err_msg=err)
                    np.testing.assert_array_equal(outs[1], want, err_msg=err)
    finally:
        lib.morph_set_composite_kernel(-1)
    # the default form: one launch for a 5 x 5 gradient, more for an opening
    img = synth.uniform_image(300, 200, dtype, gen=g)
    src = DeviceImage(torch, 200, 300, dtype, fill=img)
    for kind, one in ((lib.MORPH_GRADIENT, True), (lib.MORPH_OPEN, False)):
        dst = DeviceImage(torch, 200, 300, dtype)
        torch.cuda.synchronize()
        n0 = lib.morph_launch_count()
        assert lib.morph_composite(src.ptr, src.pitch, dst.ptr, dst.pitch, 300, 200, code, kind, 5, 5, 2, 2, 0) == 0
        torch.cuda.synchronize()
        assert (lib.morph_launch_count() - n0 == 1) == one
        np.testing.assert_array_equal(dst.read(), want_of(kind, img, 5, 5, 2, 2, lib))
    assert lib.morph_device_error() == 0
