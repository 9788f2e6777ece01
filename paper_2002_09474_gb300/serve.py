"""Continuous-batching request loop for erosion/dilation requests.

Requests (an image, a window, an anchor, an operation) arrive over time.  The
loop admits waiting requests in arrival order while a device-memory budget
allows their input and output bytes, groups the newly admitted ones into a
micro-batch that runs as ONE persistent kernel launch (morph_batch), and puts
consecutive micro-batches on different CUDA streams, so requests that arrive
while others are on the GPU start without waiting for them.  Completions are
found by polling CUDA events; a completed request frees its budget and its
output buffer goes back to a pool for reuse.  Latency is arrival to
completion.

With ``GpuExecutor`` inputs are pre-staged in device memory (requests point
into a resident source pool), so host-to-device copies are not part of the
latency; the budget still charges each request its input bytes as if
staged, its output buffer and the library's scratch (an intermediate image
for a 2-D window).  With ``HostCopyExecutor`` requests hold pinned HOST
images (dense, as a client's own buffer would be): each micro-batch's stream
copies its inputs to device buffers, runs the batch and copies the results
back to pinned host buffers, so the latency (arrival to the results in host
memory) includes both copies, and the copies of one micro-batch overlap the
filtering of others on the other streams.

The scheduling logic is independent of CUDA: it talks to an executor
(``GpuExecutor`` here; tests use a host-only fake).
"""
from __future__ import annotations

import collections
import gc
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    width: int
    height: int
    wx: int
    wy: int
    ax: int
    ay: int
    op: int
    dtype_size: int = 1           # bytes per pixel (1: u8, 2: u16)
    src: object = None            # executor-specific input handle (pre-staged)
    origin: tuple = (0, 0)        # (x0, y0) of the input in its source pool
    offset: int = -1              # or, for a dense image in a host arena, its byte offset
    # filled by the server
    admitted_s: float = -1.0
    done_s: float = -1.0
    out: object = None
    charge_bytes: int = -1        # budget charge (computed once, at arrival)
    batch_bytes: int = -1         # bytes it adds to a micro-batch

    @property
    def nbytes(self) -> int:
        """Input plus output image bytes (the default budget charge)."""
        return 2 * self.width * self.height * self.dtype_size


@dataclass
class ServeStats:
    completed: int = 0
    rejected: int = 0
    pixels: int = 0
    wall_s: float = 0.0
    latencies_ms: list = field(default_factory=list)
    max_budget_used: int = 0
    batches: int = 0
    max_in_flight: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"completed": self.completed, "rejected": self.rejected,
                "throughput_req_s": self.completed / self.wall_s if self.wall_s else 0.0,
                "gpix_s": self.pixels / self.wall_s / 1e9 if self.wall_s else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_budget_used_bytes": self.max_budget_used, "batches": self.batches,
                "max_batches_in_flight": self.max_in_flight}


class Budget:
    """Device-byte accounting for admission."""

    def __init__(self, limit: int):
        self.limit = int(limit)
        self.used = 0

    def try_take(self, n: int) -> bool:
        if self.used + n > self.limit:
            return False
        self.used += n
        return True

    def give(self, n: int) -> None:
        self.used -= n
        assert self.used >= 0


class Server:
    """The scheduling loop.  ``executor`` provides: ``n_streams``;
    ``alloc_out(req)`` -> output handle; ``launch(reqs, stream_index)`` ->
    completion token; ``done(token)`` -> bool (non-blocking);
    ``finish(req)``, called once per completed request (releases its output);
    ``idle_wait()``, a short pause while work is in flight."""

    def __init__(self, executor, budget_bytes: int = 4 << 30, max_batch: int = 128,
                 max_in_flight: int = 8):
        self.ex = executor
        # bytes a request holds while admitted (executor's own rule if it has one)
        self.charge = getattr(executor, "charge", lambda r: r.nbytes)
        self.budget = Budget(budget_bytes)
        self.max_batch = max_batch
        # bytes a request adds to a micro-batch, and the cap on their sum
        self.batch_bytes = getattr(executor, "batch_bytes", lambda r: r.nbytes)
        self.batch_cap = getattr(executor, "max_batch_bytes", None)
        self.max_in_flight = max_in_flight

    def run(self, requests: list[ServeRequest], timeout_s: float = 600.0,
            clock=time.perf_counter, pause_gc: bool = True) -> ServeStats:
        """Serves ``requests`` (arrival times relative to the start) until all
        are done.  With pause_gc, Python's cyclic garbage collector is off
        for the run (reference counting still frees everything the loop
        makes): a full collection over the run's objects stalled the loop
        for about 80 ms at 20k requests/s, and the backlog it left took
        seconds to drain."""
        was = gc.isenabled()
        if pause_gc:
            gc.disable()
        try:
            return self._run(requests, timeout_s, clock)
        finally:
            if pause_gc and was:
                gc.enable()

    def _run(self, requests, timeout_s, clock) -> ServeStats:
        st = ServeStats()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque = collections.deque()
        in_flight: list = []  # (token, reqs)
        next_stream = 0
        t0 = clock()
        while pending or waiting or in_flight:
            now = clock() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop did not drain within %.0f s" % timeout_s)
            while pending and pending[0].arrival_s <= now:
                r = pending.popleft()
                r.charge_bytes = self.charge(r)
                r.batch_bytes = self.batch_bytes(r)
                if r.charge_bytes > self.budget.limit:  # can never fit: reject now
                    st.rejected += 1
                    continue
                waiting.append(r)
            # retire completed batches first: they free budget for admission
            still = []
            for token, reqs in in_flight:
                if self.ex.done(token):
                    tdone = clock() - t0
                    for r in reqs:
                        r.done_s = tdone
                        st.latencies_ms.append((tdone - r.arrival_s) * 1e3)
                        st.completed += 1
                        st.pixels += r.width * r.height
                        self.budget.give(r.charge_bytes)
                        self.ex.finish(r)
                else:
                    still.append((token, reqs))
            in_flight = still
            # admit in arrival order while the budget (and the executor's
            # micro-batch size, if it has one) allows
            batch = []
            bbytes = 0
            if len(in_flight) < self.max_in_flight:
                while (waiting and len(batch) < self.max_batch
                       and (not batch or self.batch_cap is None
                            or bbytes + waiting[0].batch_bytes <= self.batch_cap)
                       and self.budget.try_take(waiting[0].charge_bytes)):
                    bbytes += waiting[0].batch_bytes
                    r = waiting.popleft()
                    r.admitted_s = now
                    r.out = self.ex.alloc_out(r)
                    batch.append(r)
                st.max_budget_used = max(st.max_budget_used, self.budget.used)
            if batch:
                token = self.ex.launch(batch, next_stream)
                next_stream = (next_stream + 1) % self.ex.n_streams
                in_flight.append((token, batch))
                st.batches += 1
                st.max_in_flight = max(st.max_in_flight, len(in_flight))
            elif in_flight or (waiting and not pending):
                self.ex.idle_wait()
            elif pending:
                # nothing to do until the next arrival
                dt = pending[0].arrival_s - (clock() - t0)
                if dt > 0:
                    time.sleep(min(dt, 0.0005))
        st.wall_s = clock() - t0
        return st


class GpuExecutor:
    """Runs micro-batches with morph_batch on ``n_streams`` CUDA streams.
    Output buffers come from a pool of flat device buffers in power-of-two
    size classes, so a warm server allocates nothing; the pool keeps at most
    ``pool_cap`` idle bytes."""

    def __init__(self, device="cuda", n_streams: int = 4, pool_cap: int = 4 << 30):
        import torch

        from paper_2002_09474_gb300 import morph
        self.torch = torch
        self.morph = morph
        self.device = torch.device(device)
        self.n_streams = n_streams
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.free: dict = collections.defaultdict(list)
        self.pool_cap = pool_cap
        self.pooled = 0
        self.keep = None  # when a dict, finish() stores a copy of every result by rid

    @staticmethod
    def size_class(nbytes: int) -> int:
        return max(1 << 16, 1 << (int(nbytes) - 1).bit_length())

    @staticmethod
    def scratch_bytes(r: ServeRequest) -> int:
        """The library's scratch for the request: a 2-D window may run as two
        passes through an intermediate image (16-byte pitched rows)."""
        if r.wx <= 1 or r.wy <= 1:
            return 0
        return (r.width * r.dtype_size + 15) // 16 * 16 * r.height

    def charge(self, r: ServeRequest) -> int:
        """Input bytes, the output buffer's size class and the scratch."""
        n = r.width * r.height * r.dtype_size
        return n + self.size_class(n) + self.scratch_bytes(r)

    def alloc_out(self, r: ServeRequest):
        n = r.width * r.height * r.dtype_size
        c = self.size_class(n)
        if self.free[c]:
            buf = self.free[c].pop()
            self.pooled -= c
        else:
            buf = self.torch.empty(c, dtype=self.torch.uint8, device=self.device)
        v = buf[:n]
        if r.dtype_size == 2:
            v = v.view(self.torch.uint16)
        return v.view(r.height, r.width), buf

    def finish(self, r: ServeRequest) -> None:
        out, buf = r.out
        if self.keep is not None:
            # the copy runs on the current stream, which is not ordered with
            # the executor's streams: it must complete before the buffer
            # returns to the pool, or a later micro-batch may overwrite it
            self.keep[r.rid] = out.clone()
            self.torch.cuda.current_stream().synchronize()
        c = buf.numel()
        if self.pooled + c <= self.pool_cap:
            self.free[c].append(buf)
            self.pooled += c
        r.out = None

    def launch(self, reqs, stream_index: int):
        m = self.morph
        descs = (m.MorphDesc * len(reqs))()
        for d, r in zip(descs, reqs):
            src, out = r.src, r.out[0]
            d.src, d.dst = src.data_ptr(), out.data_ptr()
            d.width, d.height = r.width, r.height
            d.src_pitch = src.stride(0) * src.element_size()
            d.dst_pitch = out.stride(0) * out.element_size()
            d.wx, d.wy, d.anchor_x, d.anchor_y = r.wx, r.wy, r.ax, r.ay
            d.op = r.op
            d.dtype = m.MORPH_U8 if r.dtype_size == 1 else m.MORPH_U16
        s = self.streams[stream_index]
        rc = m.morph_batch(descs, len(reqs), s.cuda_stream)
        if rc != 0:
            raise m.MorphError("morph_batch", rc)
        ev = self.torch.cuda.Event()
        ev.record(s)
        return ev

    def done(self, ev) -> bool:
        return ev.query()

    def idle_wait(self) -> None:
        time.sleep(0.00005)


class HostCopyExecutor(GpuExecutor):
    """GpuExecutor for requests whose ``src`` is a pinned HOST image (a dense
    2-D CPU tensor).  A micro-batch takes one device block for its inputs
    and outputs and one pinned host block for the results, each request at
    a 256-byte aligned offset, from torch's caching allocators
    (device blocks on the current stream, freed only after the micro-batch's
    completion event, so their use on another stream is safe; pinned blocks
    from the host cache, warmed at construction for the block sizes a
    micro-batch of at most ``max_batch_bytes`` needs), so a warm server does
    not allocate; completion events are reused.
    ``launch`` queues on the micro-batch's stream the copies in (one
    morph_copy_batch call for all requests), the batch (morph_batch), one
    copy of the whole output block back to the host block, and the
    completion event; the blocks go back to the caches when the batch's last
    request finishes."""

    def __init__(self, device="cuda", n_streams: int = 4, pool_cap: int = 4 << 30,
                 max_batch_bytes: int = 256 << 20):
        super().__init__(device=device, n_streams=n_streams, pool_cap=pool_cap)
        self.max_batch_bytes = max_batch_bytes
        self.blocks = {}  # batch id -> [(device block, host block, event), requests not finished]
        self.next_batch = 0
        self.events = []  # completion events free for reuse
        torch = self.torch
        # the host cache keeps freed pinned blocks by power-of-two size:
        # allocate (and free) a few of every size a micro-batch may take
        warm = []
        c = 1 << 16
        while c <= 2 * max_batch_bytes:
            warm += [torch.empty(c, dtype=torch.uint8, pin_memory=True) for _ in range(2 * n_streams)]
            c *= 2
        del warm

    @staticmethod
    def _padded(r: ServeRequest) -> int:
        return (r.width * r.height * r.dtype_size + 255) // 256 * 256

    def charge(self, r: ServeRequest) -> int:
        """Device input and output bytes (256-byte padded) and the scratch."""
        return 2 * self._padded(r) + self.scratch_bytes(r)

    def batch_bytes(self, r: ServeRequest) -> int:
        """What a request adds to a micro-batch's blocks."""
        return self._padded(r)

    def alloc_out(self, r: ServeRequest):
        return None  # the micro-batch's blocks are taken in launch()

    def finish(self, r: ServeRequest) -> None:
        out, bid = r.out
        if self.keep is not None:
            self.keep[r.rid] = out.clone()  # host memory, complete at the event
        blk = self.blocks[bid]
        blk[1] -= 1
        if blk[1] == 0:
            self.events.append(blk[0][2])  # completed: its event may be recorded again
            del self.blocks[bid]
        r.out = None

    def launch(self, reqs, stream_index: int):
        m, torch = self.morph, self.torch
        s = self.streams[stream_index]
        sh = s.cuda_stream
        offs, total = [], 0
        for r in reqs:
            offs.append(total)
            total += r.batch_bytes
        # one device block (inputs, then outputs), allocated on the current
        # stream and used on s: safe because it is freed only after the
        # batch's completion event
        dblk = torch.empty(2 * total, dtype=torch.uint8, device=self.device)
        hout = torch.empty(total, dtype=torch.uint8, pin_memory=True)
        ev = self.events.pop() if self.events else torch.cuda.Event()
        bid = self.next_batch
        self.next_batch += 1
        self.blocks[bid] = [(dblk, hout, ev), len(reqs)]
        n = len(reqs)
        copies = (m.MorphCopyDesc * n)()
        descs = (m.MorphDesc * n)()
        di = dblk.data_ptr()
        do = di + total
        u16 = m.MORPH_U16
        for c, d, r, off in zip(copies, descs, reqs, offs):
            row = r.width * r.dtype_size
            c.dst, c.src, c.bytes = di + off, r.src.data_ptr(), row * r.height
            d.src, d.dst, d.width, d.height, d.src_pitch, d.dst_pitch = di + off, do + off, r.width, r.height, row, row
            d.wx, d.wy, d.anchor_x, d.anchor_y, d.op = r.wx, r.wy, r.ax, r.ay, r.op
            if r.dtype_size == 2:
                d.dtype = u16
        rc = m.morph_copy_batch(copies, n, sh)
        if rc != 0:
            raise m.MorphError("morph_copy_batch", rc)
        rc = m.morph_batch(descs, n, sh)
        if rc != 0:
            raise m.MorphError("morph_batch", rc)
        rc = m.morph_copy_2d(hout.data_ptr(), total, do, total, total, 1, sh)
        if rc != 0:
            raise m.MorphError("morph_copy_2d", rc)
        h16 = None
        for r, off in zip(reqs, offs):
            if r.dtype_size == 2:
                if h16 is None:
                    h16 = hout.view(torch.uint16)
                r.out = (h16.as_strided((r.height, r.width), (r.width, 1), off // 2), bid)
            else:
                r.out = (hout.as_strided((r.height, r.width), (r.width, 1), off), bid)
        ev.record(s)
        return ev


def host_arena(torch, nbytes: int = 256 << 20, seed: int = 6):
    """A pinned host arena of uniform u8 bytes (and its numpy copy): request
    images are dense slices of it, as a client's own image buffer would be."""
    from paper_2002_09474_gb300 import synth
    raw = synth.uniform_image(nbytes // 4096, 4096, np.uint8, seed=seed).reshape(-1)
    return raw, torch.from_numpy(raw.copy()).pin_memory()


def make_host_requests(rate_per_s: float, duration_s: float, arena_np, arena_pinned, seed: int = 6,
                       area_hi: int = 4096 * 4096) -> list[ServeRequest]:
    """The serving workload of make_requests with pinned host inputs: each
    request's image is a dense (pitch = width) slice of the arena at a seeded
    offset."""
    from paper_2002_09474_gb300 import synth
    specs = synth.serving_requests(rate_per_s, duration_s, seed=seed, area_hi=area_hi)
    g = synth.rng(seed + 77)
    n = arena_np.size
    out = []
    for i, s in enumerate(specs):
        w, h = min(s.width, 4096), min(s.height, 4096)
        off = int(g.integers(0, n - w * h + 1))
        out.append(ServeRequest(i, s.arrival_s, w, h, s.wx, s.wy, s.ax, s.ay, s.op, 1,
                                src=arena_pinned[off:off + w * h].view(h, w), offset=off))
    return out


def request_image(r: ServeRequest, pool_img) -> np.ndarray:
    """The request's input as a numpy image (from the numpy copy of its
    source pool or arena)."""
    if r.offset >= 0:
        return pool_img[r.offset:r.offset + r.width * r.height].reshape(r.height, r.width)
    x0, y0 = r.origin
    return pool_img[y0:y0 + r.height, x0:x0 + r.width]


def source_pool(torch, width: int = 4096, height: int = 4096, seed: int = 6, device="cuda"):
    """A resident uniform u8 image that requests take windows of (pre-staged
    inputs)."""
    from paper_2002_09474_gb300 import synth
    img = synth.uniform_image(width, height, np.uint8, seed=seed)
    return img, torch.from_numpy(img).to(device)


def make_requests(rate_per_s: float, duration_s: float, pool_img, pool_dev, seed: int = 6,
                  area_hi: int = 4096 * 4096) -> list[ServeRequest]:
    """The serving workload: Poisson arrivals, log-uniform areas and aspect
    ratios, windows 1..101, mixed ops; each request's input is a window of
    the resident source pool at a seeded offset."""
    from paper_2002_09474_gb300 import synth
    specs = synth.serving_requests(rate_per_s, duration_s, seed=seed, area_hi=area_hi)
    g = synth.rng(seed + 77)
    H, W = pool_img.shape
    out = []
    for i, s in enumerate(specs):
        w, h = min(s.width, W), min(s.height, H)
        x0 = int(g.integers(0, W - w + 1))
        y0 = int(g.integers(0, H - h + 1))
        out.append(ServeRequest(i, s.arrival_s, w, h, s.wx, s.wy, s.ax, s.ay, s.op, 1,
                                src=pool_dev[y0:y0 + h, x0:x0 + w], origin=(x0, y0)))
    return out
