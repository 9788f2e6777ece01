"""Host logic of the continuous-batching server, on the CPU: a fake executor
whose batches take a set time stands in for the GPU."""
import time

import pytest

from paper_2002_09474_gb300.serve import Budget, Server, ServeRequest


class FakeExecutor:
    """A batch completes ``per_px`` seconds per pixel after its launch."""

    n_streams = 3

    def __init__(self, per_px=2e-9, limit=None):
        self.per_px = per_px
        self.live = 0
        self.max_live = 0
        self.limit = limit
        self.launches = []
        self.finished = []
        self.clock = time.perf_counter

    def alloc_out(self, r):
        self.live += r.nbytes
        self.max_live = max(self.max_live, self.live)
        if self.limit is not None:
            assert self.live <= self.limit
        return ("out", r.rid)

    def launch(self, reqs, stream_index):
        t = self.clock()
        px = sum(r.width * r.height for r in reqs)
        self.launches.append((t, stream_index, [r.rid for r in reqs]))
        return t + px * self.per_px

    def done(self, token):
        return self.clock() >= token

    def finish(self, r):
        assert r.out == ("out", r.rid)
        self.live -= r.nbytes
        self.finished.append(r.rid)

    def idle_wait(self):
        time.sleep(2e-5)


def reqs(n, gap_s, side=256, big=()):
    out = []
    for i in range(n):
        s = 4096 if i in big else side
        out.append(ServeRequest(i, i * gap_s, s, s, 3, 3, 1, 1, i % 2))
    return out


def test_budget_accounting():
    b = Budget(100)
    assert b.try_take(60) and not b.try_take(41) and b.try_take(40)
    b.give(100)
    assert b.used == 0
    with pytest.raises(AssertionError):
        b.give(1)


def test_every_request_completes_once_in_arrival_order():
    ex = FakeExecutor()
    rs = reqs(400, 2e-4)
    st = Server(ex, budget_bytes=1 << 30).run(rs, timeout_s=30)
    assert st.completed == 400 and st.rejected == 0
    assert sorted(ex.finished) == list(range(400))
    admitted = [r.admitted_s for r in rs]
    assert admitted == sorted(admitted)          # first come, first admitted
    for r in rs:
        assert r.arrival_s <= r.admitted_s <= r.done_s
    assert len(st.latencies_ms) == 400 and min(st.latencies_ms) >= 0
    assert ex.live == 0


def test_continuous_batching_overlaps_batches():
    """Requests arriving while a batch runs start in a new batch, on another
    stream, before the first completes."""
    ex = FakeExecutor(per_px=2e-7)       # a 256x256 request runs ~13 ms
    rs = reqs(20, 1e-3)
    st = Server(ex, budget_bytes=1 << 30, max_in_flight=8).run(rs, timeout_s=30)
    assert st.completed == 20
    assert st.max_in_flight > 1
    streams = {s for _, s, _ in ex.launches}
    assert len(streams) > 1
    # the second launch happened before the first batch's completion time
    (t0, _, ids0), (t1, _, _) = ex.launches[0], ex.launches[1]
    assert t1 < t0 + len(ids0) * 256 * 256 * 2e-7


def test_budget_limits_bytes_in_flight():
    limit = 3 * 2 * 256 * 256            # room for three 256x256 requests
    ex = FakeExecutor(per_px=5e-8, limit=limit)
    rs = reqs(30, 0.0)                    # all arrive at once
    st = Server(ex, budget_bytes=limit, max_batch=64).run(rs, timeout_s=30)
    assert st.completed == 30
    assert ex.max_live <= limit and st.max_budget_used <= limit
    assert max(len(ids) for _, _, ids in ex.launches) <= 3


def test_request_larger_than_budget_is_rejected():
    ex = FakeExecutor()
    rs = reqs(10, 1e-4, big={4})
    st = Server(ex, budget_bytes=2 * 1024 * 1024).run(rs, timeout_s=30)
    assert st.rejected == 1 and st.completed == 9
    assert 4 not in ex.finished


def test_max_batch_respected():
    ex = FakeExecutor()
    rs = reqs(100, 0.0)
    Server(ex, budget_bytes=1 << 30, max_batch=16).run(rs, timeout_s=30)
    assert max(len(ids) for _, _, ids in ex.launches) <= 16
    assert sorted(i for _, _, ids in ex.launches for i in ids) == list(range(100))



class CappedExecutor(FakeExecutor):
    """A FakeExecutor with a micro-batch byte cap and its own charge rule,
    counting how often the server asks for each request's charge."""

    def __init__(self, cap, **kw):
        super().__init__(**kw)
        self.max_batch_bytes = cap
        self.charges = {}
        self.batch_sizes = []

    def charge(self, r):
        self.charges[r.rid] = self.charges.get(r.rid, 0) + 1
        return 3 * r.width * r.height

    def batch_bytes(self, r):
        return r.width * r.height

    def launch(self, reqs, stream_index):
        self.batch_sizes.append(sum(r.width * r.height for r in reqs))
        return super().launch(reqs, stream_index)


def test_micro_batch_byte_cap_and_charge_once():
    """Micro-batches never exceed the executor's byte cap unless a single
    request does; every request's charge is computed once."""
    ex = CappedExecutor(cap=3 * 256 * 256, per_px=2e-8)
    rs = reqs(40, 0.0, side=256, big=(7,))  # all at once: the server must split them
    st = Server(ex, budget_bytes=1 << 30).run(rs, timeout_s=60)
    assert st.completed == 40
    for b in ex.batch_sizes:
        assert b <= 3 * 256 * 256 or b == 4096 * 4096
    assert max(ex.batch_sizes) == 4096 * 4096  # the oversized request alone
    assert set(ex.charges.values()) == {1}


@pytest.mark.parametrize("enabled", [True, False])
def test_run_restores_the_collector_state(enabled):
    import gc
    was = gc.isenabled()
    try:
        (gc.enable if enabled else gc.disable)()
        Server(FakeExecutor()).run(reqs(5, 0.0), timeout_s=30)
        assert gc.isenabled() == enabled
    finally:
        (gc.enable if was else gc.disable)()
