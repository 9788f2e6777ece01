"""morph_batch_noalloc: the batched launch for callers that may not allocate
device memory (their memory belongs to another allocator or pool, or they
run where cudaMalloc's implicit synchronisation is not allowed).  Its scratch
is a fixed array inside the library; this checks, through the C ABI, that two
calls in a row give exactly the results of the allocating morph_batch.

The file name sorts last so that a stopping run has finished every other
test before this one; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import oracle
from paper_2002_09474_gb300 import synth

from gpu_util import need_cuda

pytestmark = pytest.mark.gpu
OPS = ("erode", "dilate")


def _make_batch(lib, torch, g, n, side=400):
    srcs, refs, outs, specs = [], [], [], []
    d_ref, d_out = [], []
    for _ in range(n):
        dt = (np.uint8, np.uint16)[int(g.integers(0, 2))]
        w, h = int(g.integers(1, side)), int(g.integers(1, 3 * side // 4))
        wx, wy = int(g.integers(1, 64)), int(g.integers(1, 64))
        op = int(g.integers(0, 2))
        img = synth.uniform_image(w, h, dt, gen=g)
        src = torch.from_numpy(img).cuda()
        ref = torch.full_like(src, 0x33)
        out = torch.full_like(src, 0x66)
        for dsts, t in ((d_ref, ref), (d_out, out)):
            d = lib.MorphDesc()
            d.src, d.dst, d.width, d.height = src.data_ptr(), t.data_ptr(), w, h
            d.src_pitch = d.dst_pitch = w * np.dtype(dt).itemsize
            d.wx, d.wy, d.anchor_x, d.anchor_y = wx, wy, wx // 2, wy // 2
            d.op = op
            d.dtype = lib.MORPH_U8 if dt == np.uint8 else lib.MORPH_U16
            dsts.append(d)
        srcs.append(src)
        refs.append(ref)
        outs.append(out)
        specs.append((img, wx, wy, op))
    arr_ref = (lib.MorphDesc * n)(*d_ref)
    arr_out = (lib.MorphDesc * n)(*d_out)
    return srcs, refs, outs, specs, arr_ref, arr_out


def test_no_alloc_batch_matches_allocating_batch_twice():
    torch = need_cuda()
    from paper_2002_09474_gb300 import morph as lib
    g = synth.rng(300)
    for call in range(2):  # two calls in a row share the library's scratch
        n = 40 if call == 0 else 25
        srcs, refs, outs, specs, arr_ref, arr_out = _make_batch(lib, torch, g, n)
        assert lib.morph_batch(arr_ref, n, 0) == 0
        rc = lib.morph_batch_noalloc(arr_out, n, 0)
        assert rc == 0, lib.status_string(rc)
        assert lib.morph_device_error() == 0
        for i, (ref, out, (img, wx, wy, op)) in enumerate(zip(refs, outs, specs)):
            assert torch.equal(ref, out), (call, i)
            if i < 5:  # and a few of them against the oracle directly
                np.testing.assert_array_equal(
                    out.cpu().numpy(), oracle.morph(img, wx, wy, wx // 2, wy // 2, OPS[op]))


def test_no_alloc_largest_batch_on_a_side_stream():
    """The largest accepted batch (MORPH_NOALLOC_MAX_IMAGES small images,
    which fills the fixed records to their end), on a non-default stream, two
    calls in a row, against the allocating morph_batch on the same stream."""
    torch = need_cuda()
    from paper_2002_09474_gb300 import morph as lib
    g = synth.rng(301)
    s = torch.cuda.Stream()
    n = lib.MORPH_NOALLOC_MAX_IMAGES
    for call in range(2):
        srcs, refs, outs, specs, arr_ref, arr_out = _make_batch(lib, torch, g, n, side=48)
        torch.cuda.synchronize()
        assert lib.morph_batch(arr_ref, n, s.cuda_stream) == 0
        rc = lib.morph_batch_noalloc(arr_out, n, s.cuda_stream)
        assert rc == 0, lib.status_string(rc)
        s.synchronize()
        assert lib.morph_device_error() == 0
        for i, (ref, out) in enumerate(zip(refs, outs)):
            assert torch.equal(ref, out), (call, i)
        img, wx, wy, op = specs[-1]  # the last record, against the oracle
        np.testing.assert_array_equal(outs[-1].cpu().numpy(), oracle.morph(img, wx, wy, wx // 2, wy // 2, OPS[op]))


def test_no_alloc_rejects_more_than_the_maximum():
    need_cuda()
    from paper_2002_09474_gb300 import morph as lib
    n = lib.MORPH_NOALLOC_MAX_IMAGES + 1
    arr = (lib.MorphDesc * n)()
    assert lib.morph_batch_noalloc(arr, n, 0) == -12
    assert "no-allocation" in lib.status_string(-12)
