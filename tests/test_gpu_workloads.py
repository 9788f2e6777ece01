"""Parity at the full sizes of the workloads, through the same C-ABI calls and
launch configurations the bench times.

Every output pixel is compared with the oracle's separable van
Herk/Gil-Werman checker (itself pinned to the brute-force definition by the
CPU tests), and a few thousand sampled pixels -- corners, edges and random
interior points -- with the brute-force definition of section 2 directly.
Opening/closing are two calls (erosion then dilation by the reflected
element, and the reverse).
"""
import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

from gpu_util import need_cuda

pytestmark = pytest.mark.gpu
OPS = ("erode", "dilate")


@pytest.fixture(scope="module")
def env():
    torch = need_cuda()
    from paper_2002_09474_gb300 import morph
    morph.morph_reset_tuning()
    return torch, morph


def sample_points(w, h, wx, wy, n, seed):
    g = synth.rng(seed)
    xs = list(g.integers(0, w, n)) + [0, w - 1, 0, w - 1]
    ys = list(g.integers(0, h, n)) + [0, 0, h - 1, h - 1]
    for _ in range(n // 4):  # near the borders, inside a window's reach
        xs.append(int(g.integers(0, min(w, wx + 1))))
        ys.append(int(g.integers(0, h)))
        xs.append(int(w - 1 - g.integers(0, min(w, wx + 1))))
        ys.append(int(g.integers(0, h)))
        xs.append(int(g.integers(0, w)))
        ys.append(int(g.integers(0, min(h, wy + 1))))
        xs.append(int(g.integers(0, w)))
        ys.append(int(h - 1 - g.integers(0, min(h, wy + 1))))
    return np.array(xs, np.int32), np.array(ys, np.int32)


def gpu_apply(torch, morph, src, wx, wy, ax, ay, op):
    dst = torch.empty_like(src)
    morph.apply(src, dst, wx, wy, ax, ay, op=op)
    return dst


def check(img, got, wx, wy, ax, ay, op, seed, what):
    want = oracle.sep_vhgw(img, wx, wy, ax, ay, OPS[op])
    bad = int((got != want).sum())
    assert bad == 0, "%s: %d pixels differ from the separable checker" % (what, bad)
    h, w = img.shape
    xs, ys = sample_points(w, h, wx, wy, 2000, seed)
    pts = oracle.morph_points(img, wx, wy, ax, ay, OPS[op], xs, ys)
    np.testing.assert_array_equal(got[ys, xs], pts, err_msg=what)


def test_c1_vga_erosion_3x3(env):
    torch, morph = env
    img = synth.uniform_image(640, 480, np.uint8, seed=1)
    got = gpu_apply(torch, morph, torch.from_numpy(img).cuda(), 3, 3, 1, 1, 0).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.morph(img, 3, 3, 1, 1, "erode"))


@pytest.mark.parametrize("w", [3, 7, 15, 31, 61])
def test_c2_document_image(env, w):
    torch, morph = env
    img = synth.document_image(1920, 1080, seed=2)
    src = torch.from_numpy(img).cuda()
    for op in (0, 1):
        got = gpu_apply(torch, morph, src, w, w, w // 2, w // 2, op).cpu().numpy()
        check(img, got, w, w, w // 2, w // 2, op, 10 + w, "document %dx%d %s" % (w, w, OPS[op]))
    if w == 3:  # the brute-force definition on the whole image, once
        got = gpu_apply(torch, morph, src, 3, 3, 1, 1, 0).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.morph(img, 3, 3, 1, 1, "erode"))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("kind", ["uniform", "gradient"])
def test_c3_4096_erosion_dilation(env, dtype, kind):
    torch, morph = env
    seed = 3 if dtype == np.uint8 else 4
    img = (synth.uniform_image(4096, 4096, dtype, seed=seed) if kind == "uniform"
           else synth.gradient_image(4096, 4096, dtype, seed=seed + 100))
    src = torch.from_numpy(img).cuda()
    for (wx, wy) in synth.C3_WINDOWS:
        for op in (0, 1):
            got = gpu_apply(torch, morph, src, wx, wy, wx // 2, wy // 2, op).cpu().numpy()
            check(img, got, wx, wy, wx // 2, wy // 2, op, wx * 1000 + wy + op,
                  "%s %s %dx%d %s" % (np.dtype(dtype).name, kind, wx, wy, OPS[op]))
    assert morph.morph_device_error() == 0


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_c3_4096_opening_closing(env, dtype):
    torch, morph = env
    img = synth.gradient_image(4096, 4096, dtype, seed=(3 if dtype == np.uint8 else 4) + 100)
    src = torch.from_numpy(img).cuda()
    for (wx, wy) in synth.C3_WINDOWS:
        ax, ay = wx // 2, wy // 2
        rx, ry = wx - 1 - ax, wy - 1 - ay  # reflected element's anchor
        for first, second in ((0, 1), (1, 0)):  # opening, closing
            mid = gpu_apply(torch, morph, src, wx, wy, ax, ay, first)
            got = gpu_apply(torch, morph, mid, wx, wy, rx, ry, second).cpu().numpy()
            m = oracle.sep_vhgw(img, wx, wy, ax, ay, OPS[first])
            want = oracle.sep_vhgw(m, wx, wy, rx, ry, OPS[second])
            name = "opening" if first == 0 else "closing"
            assert int((got != want).sum()) == 0, "%s %dx%d" % (name, wx, wy)
            # opening <= x <= closing, and idempotence of the GPU composition
            if first == 0:
                assert (got <= img).all()
            else:
                assert (got >= img).all()
            again = gpu_apply(torch, morph, gpu_apply(torch, morph, torch.from_numpy(got).cuda(),
                                                       wx, wy, ax, ay, first), wx, wy, rx, ry, second)
            np.testing.assert_array_equal(again.cpu().numpy(), got)
