"""Pins of the CPU oracle to facts other than itself (CPU only).

The paper prints no numeric example, so the oracle is pinned by:
* hand-worked examples of the section 2 definition (tests/golden/),
* scipy.ndimage grey minimum/maximum filters (an independent library routine
  that computes the same definition when the border is the identity),
* exhaustive binary images, where erosion/dilation reduce to bitwise AND/OR
  over the window,
* closed forms (1x1 identity, constant image, element larger than the image,
  1-D deque filter per axis),
* invariants (duality, extensivity, monotonicity, separability, transpose
  commutation, opening/closing order and idempotence),
* and agreement of three independent formulations (brute force, separable
  van Herk/Gil-Werman, monotone deque) on many tiny inputs.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _parse_golden(path):
    image, cases, cur = None, [], None
    rows_needed = 0
    dtype = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "image":
                r, c, dt = int(tok[1]), int(tok[2]), tok[3]
                dtype = {"u8": np.uint8, "u16": np.uint16}[dt]
                image = []
                cur = image
                rows_needed = r
                continue
            if tok[0] == "case":
                op, wx, wy, ax, ay = tok[1], *map(int, tok[2:6])
                cur = []
                cases.append(((op, wx, wy, ax, ay), cur))
                continue
            cur.append([int(v) for v in tok])
    img = np.array(image, dtype=dtype)
    assert img.shape[0] == rows_needed
    return img, [(k, np.array(v, dtype=dtype)) for k, v in cases]


@pytest.mark.parametrize("name", ["hand_u8.txt", "hand_u16.txt"])
def test_golden_hand_examples(name):
    img, cases = _parse_golden(os.path.join(GOLDEN, name))
    assert cases
    for (op, wx, wy, ax, ay), want in cases:
        got = oracle.morph(img, wx, wy, ax, ay, op)
        np.testing.assert_array_equal(got, want, err_msg=str((op, wx, wy, ax, ay)))
        got2 = oracle.sep_vhgw(img, wx, wy, ax, ay, op)
        np.testing.assert_array_equal(got2, want, err_msg=str((op, wx, wy, ax, ay)))


def _scipy_morph(img, wx, wy, ax, ay, op):
    ndi = pytest.importorskip("scipy.ndimage")
    ident = int(np.iinfo(img.dtype).max) if op == "erode" else 0
    # scipy centres a size-w filter on offset w//2 and shifts it left by
    # `origin`, so the window starts at x - (w//2 + origin): origin = a - w//2.
    origin = (ay - wy // 2, ax - wx // 2)
    f = ndi.minimum_filter if op == "erode" else ndi.maximum_filter
    return f(img, size=(wy, wx), origin=origin, mode="constant", cval=ident)


def test_scipy_origin_convention_on_an_impulse():
    # One dark pixel at p; erosion output is dark exactly where the window
    # [x-a, x-a+w-1] contains p, i.e. x in [p+a-w+1, p+a].
    w, p = 5, 9
    for a in range(w):
        img = np.full((1, 20), 200, np.uint8)
        img[0, p] = 3
        out = _scipy_morph(img, w, 1, a, 0, "erode")
        dark = np.nonzero(out[0] == 3)[0]
        assert list(dark) == list(range(p + a - w + 1, p + a + 1))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_oracle_matches_scipy_filters(dtype):
    g = synth.rng(11)
    for _ in range(120):
        h, w = int(g.integers(1, 24)), int(g.integers(1, 24))
        wx, wy = int(g.integers(1, 2 * w + 2)), int(g.integers(1, 2 * h + 2))
        ax, ay = int(g.integers(0, wx)), int(g.integers(0, wy))
        img = synth.uniform_image(w, h, dtype, gen=g)
        for op in ("erode", "dilate"):
            want = _scipy_morph(img, wx, wy, ax, ay, op)
            got = oracle.morph(img, wx, wy, ax, ay, op)
            np.testing.assert_array_equal(got, want, err_msg=str((h, w, wx, wy, ax, ay, op)))


def _window_masks(side, wx, wy, ax, ay):
    masks = np.zeros((side, side), dtype=np.int64)
    for y in range(side):
        for x in range(side):
            m = 0
            for yy in range(y - ay, y - ay + wy):
                for xx in range(x - ax, x - ax + wx):
                    if 0 <= xx < side and 0 <= yy < side:
                        m |= 1 << (yy * side + xx)
            masks[y, x] = m
    return masks


@pytest.mark.parametrize("wx,wy,ax,ay", [(3, 3, 1, 1), (2, 3, 0, 2), (4, 1, 3, 0), (1, 2, 0, 0), (5, 4, 2, 1)])
def test_exhaustive_binary_4x4(wx, wy, ax, ay):
    """On {0,255} images erosion is AND and dilation is OR over the window."""
    side = 4
    masks = _window_masks(side, wx, wy, ax, ay)
    codes = np.arange(1 << 16, dtype=np.int64)
    # all images, bit (y*4+x) set = pixel 255
    bits = ((codes[:, None] >> np.arange(16)[None, :]) & 1).astype(np.uint8)
    imgs = (bits * 255).reshape(-1, side, side)
    # stack every image in one tall image with identity rows in between so
    # no window reaches a neighbour: erosion pads with 255, dilation with 0.
    gap = wy
    for op, pad in (("erode", 255), ("dilate", 0)):
        n = imgs.shape[0]
        tall = np.full((n * (side + gap), side), pad, np.uint8)
        view = tall.reshape(n, side + gap, side)
        view[:, :side, :] = imgs
        out = oracle.morph(tall, wx, wy, ax, ay, op).reshape(n, side + gap, side)[:, :side, :]
        for y in range(side):
            for x in range(side):
                m = masks[y, x]
                if op == "erode":
                    want = ((codes & m) == m)
                else:
                    want = ((codes & m) != 0)
                np.testing.assert_array_equal(out[:, y, x] == 255, want,
                                              err_msg=str((op, x, y)))


def test_exhaustive_binary_4x4_separately_for_a_sample():
    """The stacked run above relies on identity padding; check a sample of
    the binary images one call at a time as well."""
    side, (wx, wy, ax, ay) = 4, (3, 2, 1, 0)
    masks = _window_masks(side, wx, wy, ax, ay)
    g = synth.rng(12)
    for code in g.integers(0, 1 << 16, size=300):
        img = ((int(code) >> np.arange(16)) & 1).astype(np.uint8).reshape(side, side) * 255
        e = oracle.morph(img, wx, wy, ax, ay, "erode")
        d = oracle.morph(img, wx, wy, ax, ay, "dilate")
        for y in range(side):
            for x in range(side):
                m = int(masks[y, x])
                assert (e[y, x] == 255) == ((int(code) & m) == m)
                assert (d[y, x] == 255) == ((int(code) & m) != 0)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_closed_forms(dtype):
    g = synth.rng(13)
    img = synth.uniform_image(37, 23, dtype, gen=g)
    mx = int(np.iinfo(dtype).max)
    # 1x1 element is the identity
    for op in ("erode", "dilate"):
        np.testing.assert_array_equal(oracle.morph(img, 1, 1, 0, 0, op), img)
    # constant image is a fixed point
    c = np.full((11, 13), mx // 3, dtype)
    for op in ("erode", "dilate"):
        np.testing.assert_array_equal(oracle.morph(c, 7, 5, 2, 4, op), c)
    # element covering the image from every pixel: global min / max
    h, w = img.shape
    e = oracle.morph(img, 2 * w - 1, 2 * h - 1, w - 1, h - 1, "erode")
    d = oracle.morph(img, 2 * w - 1, 2 * h - 1, w - 1, h - 1, "dilate")
    assert (e == img.min()).all() and (d == img.max()).all()
    # wx x 1 and 1 x wy reduce to the 1-D sliding filter (deque) per line
    for (wx, ax) in ((1, 0), (4, 1), (9, 8), (40, 3)):
        want = np.stack([oracle.line_wedge(r, wx, ax, "erode") for r in img.astype(np.uint32)])
        np.testing.assert_array_equal(oracle.morph(img, wx, 1, ax, 0, "erode"), want.astype(dtype))
    for (wy, ay) in ((2, 0), (7, 3), (30, 29)):
        want = np.stack([oracle.line_wedge(c, wy, ay, "dilate") for c in img.T.astype(np.uint32)]).T
        np.testing.assert_array_equal(oracle.morph(img, 1, wy, 0, ay, "dilate"), want.astype(dtype))


def test_line_wedge_against_python_brute_force():
    g = synth.rng(14)
    for _ in range(200):
        n = int(g.integers(1, 30))
        w = int(g.integers(1, 2 * n + 2))
        a = int(g.integers(0, w))
        line = g.integers(0, 256, size=n)
        for op, f in (("erode", min), ("dilate", max)):
            want = [f(line[max(x - a, 0):min(x - a + w, n)]) for x in range(n)]
            np.testing.assert_array_equal(oracle.line_wedge(line, w, a, op), want)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_three_formulations_agree_on_tiny_images(dtype):
    g = synth.rng(15 + (dtype == np.uint16))
    for _ in range(150):
        h, w = int(g.integers(1, 41)), int(g.integers(1, 41))
        wx, wy = int(g.integers(1, 2 * w + 2)), int(g.integers(1, 2 * h + 2))
        ax, ay = int(g.integers(0, wx)), int(g.integers(0, wy))
        img = synth.uniform_image(w, h, dtype, gen=g)
        for op in ("erode", "dilate"):
            b1 = oracle.morph(img, wx, wy, ax, ay, op)
            b2 = oracle.sep_vhgw(img, wx, wy, ax, ay, op)
            b3 = oracle.wedge_separable(img, wx, wy, ax, ay, op)
            np.testing.assert_array_equal(b1, b2)
            np.testing.assert_array_equal(b1, b3)


def test_all_windows_and_anchors_small_sides():
    g = synth.rng(17)
    for side_w, side_h in ((1, 1), (1, 5), (6, 1), (3, 4), (5, 5)):
        img = synth.uniform_image(side_w, side_h, np.uint8, gen=g)
        for wx in range(1, 2 * side_w + 2):
            for wy in range(1, 2 * side_h + 2):
                for ax, ay in itertools.product(range(wx), range(wy)):
                    want = _scipy_morph(img, wx, wy, ax, ay, "erode")
                    np.testing.assert_array_equal(oracle.morph(img, wx, wy, ax, ay, "erode"), want)
                    np.testing.assert_array_equal(oracle.sep_vhgw(img, wx, wy, ax, ay, "erode"), want)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_invariants(dtype):
    g = synth.rng(18)
    mx = np.iinfo(dtype).max
    for _ in range(25):
        h, w = int(g.integers(1, 30)), int(g.integers(1, 30))
        wx, wy = int(g.integers(1, 12)), int(g.integers(1, 12))
        ax, ay = int(g.integers(0, wx)), int(g.integers(0, wy))
        x = synth.uniform_image(w, h, dtype, gen=g)
        e = oracle.morph(x, wx, wy, ax, ay, "erode")
        d = oracle.morph(x, wx, wy, ax, ay, "dilate")
        # duality: dilate(x) = M - erode(M - x), same element
        np.testing.assert_array_equal(d, mx - oracle.morph(mx - x, wx, wy, ax, ay, "erode"))
        # extensivity (0 <= a < w puts the pixel itself in its window)
        assert (d >= x).all() and (x >= e).all()
        # monotonicity: x <= y  =>  erode(x) <= erode(y)
        y = np.maximum(x, synth.uniform_image(w, h, dtype, gen=g))
        assert (oracle.morph(y, wx, wy, ax, ay, "erode") >= e).all()
        # separability: 2-D element = wx x 1 then 1 x wy, in either order
        sx = oracle.morph(x, wx, 1, ax, 0, "erode")
        np.testing.assert_array_equal(e, oracle.morph(sx, 1, wy, 0, ay, "erode"))
        sy = oracle.morph(x, 1, wy, 0, ay, "erode")
        np.testing.assert_array_equal(e, oracle.morph(sy, wx, 1, ax, 0, "erode"))
        # transposition swaps the element's axes
        np.testing.assert_array_equal(oracle.morph(x.T.copy(), wy, wx, ay, ax, "erode"), e.T)
        # opening <= x <= closing, both idempotent (reflected anchor)
        o = oracle.opening(x, wx, wy, ax, ay)
        c = oracle.closing(x, wx, wy, ax, ay)
        assert (o <= x).all() and (x <= c).all()
        np.testing.assert_array_equal(oracle.opening(o, wx, wy, ax, ay), o)
        np.testing.assert_array_equal(oracle.closing(c, wx, wy, ax, ay), c)


def test_same_anchor_opening_not_idempotent_for_even_window():
    """Reading of the paper's silence on the dilation's element: only the
    reflected element makes the opening idempotent for even windows; with the
    same anchor on both steps a one-pixel shift remains."""
    g = synth.rng(19)
    found = False
    for _ in range(50):
        x = synth.uniform_image(12, 1, np.uint8, gen=g)
        e = oracle.morph(x, 2, 1, 1, 0, "erode")
        o_same = oracle.morph(e, 2, 1, 1, 0, "dilate")
        if not np.array_equal(oracle.morph(oracle.morph(o_same, 2, 1, 1, 0, "erode"), 2, 1, 1, 0, "dilate"), o_same):
            found = True
            break
    assert found


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_transpose(dtype):
    g = synth.rng(20)
    for (h, w) in ((1, 1), (8, 8), (16, 16), (5, 37), (33, 2)):
        x = synth.uniform_image(w, h, dtype, gen=g)
        t = oracle.transpose(x)
        assert t.shape == (w, h)
        assert all(t[j, i] == x[i, j] for i in range(h) for j in range(w))
        np.testing.assert_array_equal(oracle.transpose(t), x)


def test_points_equal_full_image():
    g = synth.rng(21)
    img = synth.uniform_image(50, 31, np.uint16, gen=g)
    full = oracle.morph(img, 9, 4, 3, 0, "dilate")
    xs = g.integers(0, 50, size=400)
    ys = g.integers(0, 31, size=400)
    pts = oracle.morph_points(img, 9, 4, 3, 0, "dilate", xs, ys)
    np.testing.assert_array_equal(pts, full[ys, xs])


def test_pitched_source_is_respected():
    g = synth.rng(22)
    big = synth.uniform_image(40, 9, np.uint8, gen=g)
    view = big[:, 3:29]  # non-contiguous: the wrapper copies to a dense image
    np.testing.assert_array_equal(oracle.morph(view, 5, 3, 2, 1, "erode"),
                                  oracle.morph(view.copy(), 5, 3, 2, 1, "erode"))


def test_bad_arguments_rejected():
    img = np.zeros((4, 4), np.uint8)
    for args in ((0, 1, 0, 0), (1, 0, 0, 0), (3, 3, 3, 0), (3, 3, 0, 3), (3, 3, -1, 0)):
        with pytest.raises(ValueError):
            oracle.morph(img, *args, op="erode")


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_gradient_against_window_range_brute_force(dtype):
    """The gradient is the range (max - min) of each pixel's clipped window,
    written out here in plain Python loops; constant images and 1 x 1 windows
    give 0; it never exceeds the type's range."""
    g = synth.rng(901)
    hi = np.iinfo(dtype).max
    for _ in range(12):
        h, w = int(g.integers(1, 9)), int(g.integers(1, 9))
        wx, wy = int(g.integers(1, 2 * w + 2)), int(g.integers(1, 2 * h + 2))
        ax, ay = int(g.integers(0, wx)), int(g.integers(0, wy))
        x = g.integers(0, hi + 1, size=(h, w)).astype(dtype)
        want = np.zeros_like(x)
        for y in range(h):
            for xx in range(w):
                cells = [int(x[v, u]) for v in range(y - ay, y - ay + wy) for u in range(xx - ax, xx - ax + wx)
                         if 0 <= v < h and 0 <= u < w]
                want[y, xx] = max(cells) - min(cells)
        np.testing.assert_array_equal(oracle.gradient(x, wx, wy, ax, ay), want)
    c = np.full((7, 5), 3 if dtype == np.uint8 else 40000, dtype)
    np.testing.assert_array_equal(oracle.gradient(c, 3, 5), np.zeros_like(c))
    x = g.integers(0, hi + 1, size=(6, 6)).astype(dtype)
    np.testing.assert_array_equal(oracle.gradient(x, 1, 1), np.zeros_like(x))
