"""The batched and served forms at their full workload sizes: 2000 uneven
images in one CUDA-graph launch, and a Poisson request stream through the
continuous-batching server.  Each result must equal the same image filtered
alone (one morph_apply call), and a seeded sample is checked against the
oracle."""
import ctypes

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


def check_sample(img, got, wx, wy, ax, ay, op, seed):
    np.testing.assert_array_equal(got, oracle.sep_vhgw(img, wx, wy, ax, ay, OPS[op]))
    g = synth.rng(seed)
    h, w = img.shape
    xs = np.concatenate([g.integers(0, w, 200), [0, w - 1]]).astype(np.int32)
    ys = np.concatenate([g.integers(0, h, 200), [h - 1, 0]]).astype(np.int32)
    np.testing.assert_array_equal(got[ys, xs], oracle.morph_points(img, wx, wy, ax, ay, OPS[op], xs, ys))


def test_batch_every_form(env):
    """One batch whose images take every form: the fused kernel (direct-method
    windows, small images), the pass along x alone (wx x 1), the pass along y
    alone (1 x wy), and both through an intermediate (2-D windows above the
    crossovers) -- u8 and u16, tight and padded pitches, anchor extremes --
    each compared with the oracle, through morph_batch and the graph plan.
    Sources and destinations start at offsets of 0-2 pixels from an aligned
    address, with pitches aligned or not: a 2-D window whose source rows the
    pass-along-x kernel cannot load runs its pass along y first."""
    torch, morph = env
    g = synth.rng(71)
    cases = []
    for dt in (np.uint8, np.uint16):
        esz = np.dtype(dt).itemsize
        for (w, h) in ((300, 200), (257, 129), (64, 40), (1000, 33), (130, 700), (5, 3)):
            for (wx, wy) in ((3, 3), (1, 51), (51, 1), (21, 51), (127, 127), (9, 200), (40, 9), (17, 1), (5, 40),
                             (3, 90)):
                ax, ay = [int(g.integers(0, k)) for k in (wx, wy)]
                op = int(g.integers(0, 2))
                pad = (16 - (w * esz) % 16) % 16 if (w + wx) % 2 else 3 * esz
                so, do = [esz * int(g.integers(0, 3)) for _ in range(2)]
                cases.append((dt, w, h, wx, wy, ax, ay, op, pad, so, do))
    imgs, srcs, outs = [], [], []
    arr = (morph.MorphDesc * len(cases))()
    for d, (dt, w, h, wx, wy, ax, ay, op, pad, so, do) in zip(arr, cases):
        esz = np.dtype(dt).itemsize
        img = synth.uniform_image(w, h, dt, gen=g)
        pitch = w * esz + pad
        src = torch.zeros(h * pitch + 64, dtype=torch.uint8, device="cuda")
        view = src[so:so + h * pitch].view(h, pitch)[:, :w * esz]
        view.copy_(torch.from_numpy(img.view(np.uint8).reshape(h, w * esz)).cuda())
        out = torch.full((h * pitch + 64,), 0x5A, dtype=torch.uint8, device="cuda")
        d.src, d.dst, d.width, d.height = src.data_ptr() + so, out.data_ptr() + do, w, h
        d.src_pitch = d.dst_pitch = pitch
        d.wx, d.wy, d.anchor_x, d.anchor_y, d.op = wx, wy, ax, ay, op
        d.dtype = morph.MORPH_U8 if dt == np.uint8 else morph.MORPH_U16
        imgs.append(img)
        srcs.append(src)
        outs.append(out)

    def check():
        torch.cuda.synchronize()
        assert morph.morph_device_error() == 0
        for (dt, w, h, wx, wy, ax, ay, op, pad, so, do), img, out in zip(cases, imgs, outs):
            esz = np.dtype(dt).itemsize
            pitch = w * esz + pad
            host = out.cpu().numpy()
            got = host[do:do + h * pitch].reshape(h, pitch)[:, :w * esz].copy().view(dt)
            want = oracle.morph(img, wx, wy, ax, ay, OPS[op])
            assert np.array_equal(got, want), (dt.__name__, w, h, wx, wy, ax, ay, op, pad, so, do)
            rest = host[do:do + h * pitch].reshape(h, pitch)[:, w * esz:]
            assert (rest == 0x5A).all() and (host[do + h * pitch:] == 0x5A).all() and (host[:do] == 0x5A).all(), \
                "wrote outside the image"
            out.fill_(0x5A)

    assert morph.morph_batch(arr, len(cases), 0) == 0
    check()
    plan = ctypes.c_void_p()
    rc = morph.morph_batch_plan_create(arr, len(cases), ctypes.byref(plan))
    assert rc == 0, morph.status_string(rc)
    try:
        for _ in range(2):
            assert morph.morph_batch_plan_launch(plan, 0) == 0
            check()
    finally:
        assert morph.morph_batch_plan_destroy(plan) == 0


def test_batch_two_pass_forms_on_large_images(env):
    """2-D windows above the crossovers on images of 2 Mpixels: with source
    rows the batched pass-along-x kernel can load, the image takes the
    batched two-pass form; otherwise (unaligned base or pitch) it runs as
    its single call.  Either way a single-image batch is two launches,
    equals the single call, and matches the oracle (the separable checker in
    full, the brute force at sample points)."""
    torch, morph = env
    g = synth.rng(72)
    cases = [(np.uint8, 1536, 1400, 21, 51, 0, 0), (np.uint8, 1537, 1400, 21, 51, 1, 3),
             (np.uint16, 1500, 1450, 99, 37, 0, 0), (np.uint16, 1501, 1450, 99, 37, 2, 6)]
    _two_pass_cases(torch, morph, g, cases)


def _two_pass_cases(torch, morph, g, cases):
    for k, (dt, w, h, wx, wy, so, do) in enumerate(cases):
        esz = np.dtype(dt).itemsize
        img = synth.uniform_image(w, h, dt, gen=g)
        pitch = w * esz
        src = torch.zeros(h * pitch + 64, dtype=torch.uint8, device="cuda")
        src[so:so + h * pitch].copy_(torch.from_numpy(img.view(np.uint8).reshape(-1)).cuda())
        outs = [torch.full((h * pitch + 64,), 0x5A, dtype=torch.uint8, device="cuda") for _ in range(2)]
        ax, ay, op = wx // 3, wy - 1, k % 2
        dtype = morph.MORPH_U8 if dt == np.uint8 else morph.MORPH_U16
        d = morph.MorphDesc()
        d.src, d.dst, d.width, d.height = src.data_ptr() + so, outs[0].data_ptr() + do, w, h
        d.src_pitch = d.dst_pitch = pitch
        d.wx, d.wy, d.anchor_x, d.anchor_y, d.op, d.dtype = wx, wy, ax, ay, op, dtype
        torch.cuda.synchronize()
        n0 = morph.morph_launch_count()
        assert morph.morph_batch((morph.MorphDesc * 1)(d), 1, 0) == 0
        assert morph.morph_launch_count() - n0 == 2, "not the two-pass form"
        assert morph.morph_apply(src.data_ptr() + so, pitch, outs[1].data_ptr() + do, pitch, w, h, dtype, op,
                                 wx, wy, ax, ay, 0) == 0
        torch.cuda.synchronize()
        assert morph.morph_device_error() == 0
        assert torch.equal(outs[0], outs[1])
        host = outs[0].cpu().numpy()
        assert (host[:do] == 0x5A).all() and (host[do + h * pitch:] == 0x5A).all()
        got = host[do:do + h * pitch].copy().view(dt).reshape(h, w)
        check_sample(img, got, wx, wy, ax, ay, op, seed=720 + k)


def test_batch_2000_images_graph_plan(env):
    torch, morph = env
    specs = synth.batch_specs(2000, seed=5)
    pix = synth.batch_pixels(specs, seed=5)
    srcs = [torch.from_numpy(p).cuda() for p in pix]
    outs = [torch.full_like(s, 0x5A) for s in srcs]
    arr = (morph.MorphDesc * len(specs))()
    for d, s, o, sp in zip(arr, srcs, outs, specs):
        d.src, d.dst, d.width, d.height = s.data_ptr(), o.data_ptr(), sp.width, sp.height
        d.src_pitch = d.dst_pitch = sp.width
        d.wx, d.wy, d.anchor_x, d.anchor_y, d.op = sp.wx, sp.wy, sp.ax, sp.ay, sp.op
        d.dtype = morph.MORPH_U8
    plan = ctypes.c_void_p()
    rc = morph.morph_batch_plan_create(arr, len(specs), ctypes.byref(plan))
    assert rc == 0, morph.status_string(rc)
    try:
        for rep in range(2):  # the graph replays to the same result
            rc = morph.morph_batch_plan_launch(plan, 0)
            assert rc == 0, morph.status_string(rc)
            torch.cuda.synchronize()
            assert morph.morph_device_error() == 0
            alone = torch.empty(2048 * 2048, dtype=torch.uint8, device="cuda")
            for i, (s, o, sp) in enumerate(zip(srcs, outs, specs)):
                a = alone[:sp.width * sp.height].view(sp.height, sp.width)
                morph.apply(s, a, sp.wx, sp.wy, sp.ax, sp.ay, op=sp.op)
                assert torch.equal(a, o), (i, sp)
            for o in outs:
                o.fill_(0x5A)
    finally:
        assert morph.morph_batch_plan_destroy(plan) == 0
    # a seeded sample of 64 images against the oracle (after one more replay)
    assert morph.morph_batch(arr, len(specs), 0) == 0
    torch.cuda.synchronize()
    for i in synth.rng(55).choice(len(specs), 64, replace=False):
        sp = specs[i]
        check_sample(pix[i], outs[i].cpu().numpy(), sp.wx, sp.wy, sp.ax, sp.ay, sp.op, 500 + int(i))


def test_serving_results_equal_alone(env):
    """Poisson stream at 5k req/s, full area range, 4 GB budget: every
    request's result equals the same request run alone, and a sample equals
    the oracle."""
    torch, morph = env
    from paper_2002_09474_gb300 import serve
    pool_img, pool_dev = serve.source_pool(torch, seed=6)
    rs = serve.make_requests(5000.0, 0.12, pool_img, pool_dev, seed=6)
    assert len(rs) > 300
    ex = serve.GpuExecutor(n_streams=4)
    ex.keep = {}
    st = serve.Server(ex, budget_bytes=4 << 30).run(rs, timeout_s=120)
    torch.cuda.synchronize()
    assert morph.morph_device_error() == 0
    assert st.completed == len(rs) and st.rejected == 0 and st.batches > 1
    assert st.max_budget_used <= 4 << 30
    for r in rs:
        alone = torch.empty((r.height, r.width), dtype=torch.uint8, device="cuda")
        morph.apply(r.src, alone, r.wx, r.wy, r.ax, r.ay, op=r.op)
        assert torch.equal(alone, ex.keep[r.rid]), r
    for i in synth.rng(66).choice(len(rs), 24, replace=False):
        r = rs[int(i)]
        x0, y0 = r.origin
        img = pool_img[y0:y0 + r.height, x0:x0 + r.width]
        check_sample(img, ex.keep[r.rid].cpu().numpy(), r.wx, r.wy, r.ax, r.ay, r.op, 700 + int(i))


def test_serving_budget_binds(env):
    """A budget that holds only a few requests still drains the stream, never
    holds more than it allows, and gives the same results."""
    torch, morph = env
    from paper_2002_09474_gb300 import serve
    pool_img, pool_dev = serve.source_pool(torch, seed=7)
    rs = serve.make_requests(20000.0, 0.01, pool_img, pool_dev, seed=7, area_hi=1024 * 1024)
    ex = serve.GpuExecutor(n_streams=2)
    ex.keep = {}
    budget = 3 * ex.charge(max(rs, key=ex.charge))
    st = serve.Server(ex, budget_bytes=budget).run(rs, timeout_s=60)
    torch.cuda.synchronize()
    assert st.completed == len(rs) and st.max_budget_used <= budget
    for r in rs:
        alone = torch.empty((r.height, r.width), dtype=torch.uint8, device="cuda")
        morph.apply(r.src, alone, r.wx, r.wy, r.ax, r.ay, op=r.op)
        assert torch.equal(alone, ex.keep[r.rid]), r


def test_serving_with_host_copies(env):
    """Requests hold pinned host images; each micro-batch copies its inputs
    in, filters and copies the results back on its stream: every result (in
    host memory) equals the request run alone on the device, a sample equals
    the oracle, and the budget (device input and output buffers) holds."""
    torch, morph = env
    from paper_2002_09474_gb300 import serve
    pool_img, pool_host = serve.host_arena(torch, seed=8)
    rs = serve.make_host_requests(3000.0, 0.1, pool_img, pool_host, seed=8)
    assert len(rs) > 150
    ex = serve.HostCopyExecutor(n_streams=4)
    ex.keep = {}
    budget = 2 << 30
    st = serve.Server(ex, budget_bytes=budget).run(rs, timeout_s=120)
    torch.cuda.synchronize()
    assert morph.morph_device_error() == 0
    assert st.completed == len(rs) and st.rejected == 0 and st.batches > 1
    assert st.max_budget_used <= budget
    for r in rs:
        res = ex.keep[r.rid]
        assert not res.is_cuda
        src = r.src.cuda()
        alone = torch.empty_like(src)
        morph.apply(src, alone, r.wx, r.wy, r.ax, r.ay, op=r.op)
        assert torch.equal(alone.cpu(), res), r
    for i in synth.rng(88).choice(len(rs), 16, replace=False):
        r = rs[int(i)]
        img = serve.request_image(r, pool_img)
        check_sample(img, ex.keep[r.rid].numpy(), r.wx, r.wy, r.ax, r.ay, r.op, 800 + int(i))
