"""GPU parity of the transpose kernels (section 4), the batched persistent
launch and its CUDA-graph plan, the host-buffer entry point and the
autotuner -- all bit-exact against the CPU oracle."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

from gpu_util import DeviceImage, need_cuda

pytestmark = pytest.mark.gpu
OPS = ("erode", "dilate")


@pytest.fixture(scope="module")
def lib():
    need_cuda()
    from paper_2002_09474_gb300 import morph
    morph.morph_reset_tuning()
    yield morph
    morph.morph_reset_tuning()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_transpose(lib, dtype):
    torch = need_cuda()
    g = synth.rng(200)
    esz = np.dtype(dtype).itemsize
    fn = lib.transpose_u8 if dtype == np.uint8 else lib.transpose_u16
    for (h, w) in ((1, 1), (3, 5), (8, 8), (16, 16), (64, 64), (65, 63), (100, 257), (512, 300)):
        img = synth.uniform_image(w, h, dtype, gen=g)
        for spad, dpad in ((0, 0), ((16 - w * esz % 16) % 16, (16 - h * esz % 16) % 16), (6, 2)):
            src = DeviceImage(torch, h, w, dtype, pad=spad, fill=img)
            dst = DeviceImage(torch, w, h, dtype, pad=dpad)
            rc = fn(src.ptr, w, h, src.pitch, dst.ptr, dst.pitch, 0)
            assert rc == 0, lib.status_string(rc)
            torch.cuda.synchronize()
            assert dst.untouched_outside()
            np.testing.assert_array_equal(dst.read(), oracle.transpose(img))
            np.testing.assert_array_equal(dst.read(), img.T)


def test_transpose_commutes_with_erosion(lib):
    """erode(S^T, wy x wx) = erode(S, wx x wy)^T through the GPU path."""
    torch = need_cuda()
    img = synth.uniform_image(200, 130, np.uint8, seed=201)
    s = torch.from_numpy(img).cuda()
    t = torch.empty((200, 130), dtype=torch.uint8, device="cuda")
    lib.transpose(s, t)
    e1 = torch.empty_like(s)
    e2 = torch.empty_like(t)
    lib.apply(s, e1, 21, 5, op=0)
    lib.apply(t, e2, 5, 21, op=0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(e1.cpu().numpy().T, e2.cpu().numpy())


def _batch(lib, torch, specs, g):
    """Device images for specs (u8/u16 mixed), descriptors, and the expected
    oracle outputs."""
    imgs, outs, descs, want = [], [], [], []
    for (w, h, wx, wy, ax, ay, op, dt) in specs:
        img = synth.uniform_image(w, h, dt, gen=g)
        src = torch.from_numpy(img).cuda()
        dst = torch.full_like(src, 0x5A)
        imgs.append(src)
        outs.append(dst)
        d = lib.MorphDesc()
        d.src, d.dst, d.width, d.height = src.data_ptr(), dst.data_ptr(), w, h
        d.src_pitch = d.dst_pitch = w * np.dtype(dt).itemsize
        d.wx, d.wy, d.anchor_x, d.anchor_y = wx, wy, ax, ay
        d.op = op
        d.dtype = lib.MORPH_U8 if dt == np.uint8 else lib.MORPH_U16
        descs.append(d)
        want.append(oracle.morph(img, wx, wy, ax, ay, OPS[op]))
    arr = (lib.MorphDesc * len(descs))(*descs)
    return imgs, outs, arr, want


def _random_specs(g, n, side_hi=300, w_hi=63, dtypes=(np.uint8, np.uint16)):
    specs = []
    for _ in range(n):
        w, h = int(g.integers(1, side_hi)), int(g.integers(1, side_hi))
        wx, wy = int(g.integers(1, w_hi + 1)), int(g.integers(1, w_hi + 1))
        specs.append((w, h, wx, wy, wx // 2, wy // 2, int(g.integers(0, 2)),
                      dtypes[int(g.integers(0, len(dtypes)))]))
    return specs


def test_batch_single_launch(lib):
    torch = need_cuda()
    g = synth.rng(210)
    specs = _random_specs(g, 60) + [(1, 1, 1, 1, 0, 0, 0, np.uint8), (2048, 3, 63, 1, 31, 0, 1, np.uint8),
                                     (3, 700, 1, 63, 0, 31, 0, np.uint16)]
    imgs, outs, arr, want = _batch(lib, torch, specs, g)
    rc = lib.morph_batch(arr, len(specs), 0)
    assert rc == 0, lib.status_string(rc)
    assert lib.morph_device_error() == 0
    for i, (o, w) in enumerate(zip(outs, want)):
        np.testing.assert_array_equal(o.cpu().numpy(), w, err_msg=str(specs[i]))


def test_batch_plan_graph_replays(lib):
    torch = need_cuda()
    g = synth.rng(211)
    specs = _random_specs(g, 40)
    imgs, outs, arr, want = _batch(lib, torch, specs, g)
    plan = ctypes.c_void_p()
    rc = lib.morph_batch_plan_create(arr, len(specs), ctypes.byref(plan))
    assert rc == 0, lib.status_string(rc)
    try:
        for _ in range(3):
            for o in outs:
                o.fill_(0x5A)
            rc = lib.morph_batch_plan_launch(plan, 0)
            assert rc == 0, lib.status_string(rc)
            assert lib.morph_device_error() == 0
            for i, (o, w) in enumerate(zip(outs, want)):
                np.testing.assert_array_equal(o.cpu().numpy(), w, err_msg=str(specs[i]))
    finally:
        assert lib.morph_batch_plan_destroy(plan) == 0


def test_batch_matches_single_calls(lib):
    """Each image's batched result equals its single-image result."""
    torch = need_cuda()
    g = synth.rng(212)
    specs = [s for s in _random_specs(g, 30, side_hi=600, dtypes=(np.uint8,))]
    imgs, outs, arr, want = _batch(lib, torch, specs, g)
    assert lib.morph_batch(arr, len(specs), 0) == 0
    for (w, h, wx, wy, ax, ay, op, dt), src, o in zip(specs, imgs, outs):
        single = torch.empty_like(src)
        lib.apply(src, single, wx, wy, ax, ay, op=op)
        torch.cuda.synchronize()
        assert torch.equal(single, o)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_host_buffer_entry_point(lib, dtype):
    torch = need_cuda()
    g = synth.rng(220)
    img = synth.uniform_image(333, 211, dtype, gen=g)
    tdt = torch.uint8 if dtype == np.uint8 else torch.uint16
    for pinned in (False, True):
        src = torch.from_numpy(img.copy())
        dst = torch.zeros((211, 333), dtype=tdt)
        if pinned:
            src, dst = src.pin_memory(), dst.pin_memory()
        for (wx, wy, op) in ((3, 3, 0), (21, 51, 1), (127, 1, 0)):
            lib.apply_host(src, dst, wx, wy, op=op)
            np.testing.assert_array_equal(dst.numpy(), oracle.morph(img, wx, wy, wx // 2, wy // 2, OPS[op]))
    assert lib.morph_release_staging() == 0


def test_autotune_and_cache(lib, tmp_path):
    torch = need_cuda()
    path = str(tmp_path / "tune.json")
    assert lib.morph_autotune(path) == 0
    text = open(path).read()
    assert '"cross"' in text and '"device"' in text and '"xpass"' in text
    assert '"rowv_rows"' in text and '"fused_cfg"' in text and '"colv_family"' in text
    # a second call loads the cache; results stay exact either way
    assert lib.morph_autotune(path) == 0
    img = synth.uniform_image(300, 200, np.uint8, seed=221)
    s = torch.from_numpy(img).cuda()
    for (wx, wy) in ((9, 9), (15, 31), (63, 5), (1, 101), (101, 1), (21, 51)):
        o = torch.empty_like(s)
        lib.apply(s, o, wx, wy, op=0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o.cpu().numpy(), oracle.morph(img, wx, wy, wx // 2, wy // 2, "erode"))
    # the measured launch shapes, on an image large enough to use them
    # (the tile heights of the pass along y in every window class, and the
    # fused tile shapes of the direct-method window classes)
    for dt in (np.uint8, np.uint16):
        big = synth.uniform_image(4000, 3300, dt, seed=222)
        s = torch.from_numpy(big).cuda()
        for (wx, wy) in ((1, 15), (1, 31), (1, 51), (1, 101), (1, 127), (101, 1), (21, 51), (127, 127),
                         (3, 3), (5, 5), (7, 7), (9, 9)):
            o = torch.empty_like(s)
            lib.apply(s, o, wx, wy, op=1)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(o.cpu().numpy(), oracle.sep_vhgw(big, wx, wy, wx // 2, wy // 2, "dilate"),
                                          err_msg="%s %dx%d" % (dt.__name__, wx, wy))
    lib.morph_reset_tuning()


def test_host_batch_pipeline_matches_single_calls(lib):
    """morph_apply_host_batch (copies in, filtering and copies out of
    consecutive images overlapped) gives every image exactly the result of
    morph_apply_host, over more images than staging slots, mixed types,
    sizes, windows and pitches, twice in a row."""
    import ctypes
    torch = need_cuda()
    g = synth.rng(620)
    imgs, outs, singles, descs = [], [], [], (lib.MorphDesc * 7)()
    for i, d in enumerate(descs):
        dt = (np.uint8, np.uint16)[i % 2]
        h, w = int(g.integers(1, 700)), int(g.integers(1, 900))
        img = synth.uniform_image(w, h, dt, gen=g)
        src = torch.from_numpy(img).pin_memory()
        out = torch.zeros_like(src).pin_memory()
        one = torch.zeros_like(src).pin_memory()
        wx, wy = int(g.integers(1, 130)), int(g.integers(1, 130))
        op = i % 2
        code = lib.MORPH_U8 if dt == np.uint8 else lib.MORPH_U16
        pitch = w * np.dtype(dt).itemsize
        rc = lib.morph_apply_host(src.data_ptr(), pitch, one.data_ptr(), pitch, w, h, code, op,
                                  wx, wy, wx // 2, wy // 2, 0)
        assert rc == 0, lib.status_string(rc)
        d.src, d.dst, d.width, d.height = src.data_ptr(), out.data_ptr(), w, h
        d.src_pitch = d.dst_pitch = pitch
        d.wx, d.wy, d.anchor_x, d.anchor_y, d.op, d.dtype = wx, wy, wx // 2, wy // 2, op, code
        imgs.append(src)
        outs.append(out)
        singles.append(one)
    for _ in range(2):
        for o in outs:
            o.zero_()
        rc = lib.morph_apply_host_batch(descs, len(descs), 0)
        assert rc == 0, lib.status_string(rc)
        for i, (o, one) in enumerate(zip(outs, singles)):
            assert torch.equal(o, one), i
    want = oracle.morph(imgs[0].numpy(), descs[0].wx, descs[0].wy, descs[0].anchor_x,
                        descs[0].anchor_y, "erode")
    assert np.array_equal(outs[0].numpy(), want)
    bad = (lib.MorphDesc * 1)()
    ctypes.memmove(ctypes.addressof(bad), ctypes.addressof(descs), ctypes.sizeof(lib.MorphDesc))
    bad[0].wx = 0
    assert lib.morph_apply_host_batch(bad, 1, 0) == -3  # MORPH_ERR_WINDOW
    lib.morph_release_staging()
    lib.check_device_error()


def test_bounded_wait_gives_up_and_context_survives(lib):
    """Failure detection on the GPU without a fault: a warp waits, bounded,
    on an mbarrier phase nothing completes; after the limit it records error
    1, which morph_device_error() reports once (then 0), and the next call on
    the same context is exact."""
    import time
    torch = need_cuda()
    assert lib.morph_device_error() == 0
    t0 = time.perf_counter()
    assert lib.morph_selftest_wait_timeout(0) == 0
    assert lib.morph_device_error() == 1  # synchronises: the wait has given up
    waited = time.perf_counter() - t0
    assert 1.5 < waited < 30.0, waited
    assert lib.morph_device_error() == 0
    img = synth.uniform_image(300, 200, np.uint8, seed=230)
    s = torch.from_numpy(img).cuda()
    o = torch.empty_like(s)
    lib.apply(s, o, 9, 7, op=0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o.cpu().numpy(), oracle.morph(img, 9, 7, 4, 3, "erode"))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_typed_entry_points(lib, dtype):
    """The typed single-image entry points (morph_erode, morph_dilate,
    morph_erode_u16, morph_dilate_u16: one pitch for source and destination)
    against the oracle, on every form a call takes: fused small windows, the
    single-pass kernels of 1-D windows, and the two-launch form of a 2-D
    window on an image of 2 Mpixels; guard bytes around the destination."""
    torch = need_cuda()
    g = synth.rng(910)
    esz = np.dtype(dtype).itemsize
    fns = {(np.uint8, "erode"): lib.morph_erode, (np.uint8, "dilate"): lib.morph_dilate,
           (np.uint16, "erode"): lib.morph_erode_u16, (np.uint16, "dilate"): lib.morph_dilate_u16}
    for (w, h, wx, wy) in ((300, 200, 3, 5), (1000, 300, 1, 101), (1000, 300, 101, 1), (2048, 1024, 21, 51),
                           (77, 33, 127, 127)):
        img = synth.uniform_image(w, h, dtype, gen=g)
        pad = (16 - (w * esz) % 16) % 16
        for op in ("erode", "dilate"):
            ax, ay = int(g.integers(0, wx)), int(g.integers(0, wy))
            src = DeviceImage(torch, h, w, dtype, pad=pad, fill=img)
            dst = DeviceImage(torch, h, w, dtype, pad=pad)
            assert src.pitch == dst.pitch
            rc = fns[(dtype, op)](src.ptr, w, h, src.pitch, wx, wy, ax, ay, dst.ptr, 0)
            assert rc == 0, lib.status_string(rc)
            torch.cuda.synchronize()
            assert lib.morph_device_error() == 0
            assert dst.untouched_outside()
            got = dst.read()
            if w * h <= 400000:
                want = oracle.morph(img, wx, wy, ax, ay, op)
            else:
                want = oracle.sep_vhgw(img, wx, wy, ax, ay, op)
                xs = g.integers(0, w, 300).astype(np.int32)
                ys = g.integers(0, h, 300).astype(np.int32)
                np.testing.assert_array_equal(got[ys, xs], oracle.morph_points(img, wx, wy, ax, ay, op, xs, ys))
            np.testing.assert_array_equal(got, want, err_msg="%s %s %dx%d %dx%d" % (dtype.__name__, op, w, h, wx, wy))
