"""The serving form's scheduler on the CPU, against a simulated GPU: fake
streams, events and octrees on a simulated clock drive the real request loop
(admission, continuous batching, frame budgets, frames, per-batch
completion). Checks: every request is applied exactly once and, per octree,
in arrival order (the gidx order the octree's contents depend on), even when
a frame budget stops a launch and its remaining requests go back to the
queue; never more persistent launches in flight than launch slots; frames
are drawn."""
import contextlib
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_03567_gb300 import serving, simlod


class Clock:
    """Simulated time: only sleeping advances it. A run that is still going
    after `limit` simulated seconds has stalled (requests that never finish
    keep their staging ranges, and admission then waits for ever): fail."""

    def __init__(self, limit=30.0):
        self.t = 0.0
        self.limit = limit

    def perf_counter(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)
        if self.t > self.limit:
            raise AssertionError("the scheduler stalled: simulated time ran out")


class FakeStream:
    def __init__(self, clock):
        self.clock = clock
        self.t_free = 0.0  # when the work enqueued so far is done

    def start(self):
        return max(self.t_free, self.clock.t)

    def wait_event(self, ev):
        self.t_free = max(self.t_free, ev.t)


class FakeEvent:
    clock = None

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = stream.start() if stream is not None else self.clock.t

    def query(self):
        return self.t is not None and self.clock.t >= self.t

    def synchronize(self):
        self.clock.t = max(self.clock.t, self.t)

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


class FakeCuda:
    def __init__(self, clock):
        FakeEvent.clock = clock
        self.Event = FakeEvent

    @staticmethod
    def stream(s):
        return contextlib.nullcontext()


class FakeTorch:
    int64 = torch.int64

    def __init__(self, clock):
        self.cuda = FakeCuda(clock)

    @staticmethod
    def empty(shape, dtype=None, device=None):
        return None


class FakeOctree:
    """Applies a launch's batches one after another at `rate` points per
    second of simulated time; with a budget, a batch after the first starts
    only while the launch has run for at most the budget (the persistent
    kernel's frame-budget rule). Records the request id each batch carries in
    its first record."""

    def __init__(self, clock, rate, render_s):
        self.clock, self.rate, self.render_s = clock, rate, render_s
        self.stream = FakeStream(clock)
        self.done_at = []   # completion time of every batch applied
        self.applied = []   # request ids in the order their batches were applied
        self.launch_spans = []

    def _apply(self, ptrs, counts, budget_ns):
        t0 = t = self.stream.start()
        for i, (p, n) in enumerate(zip(ptrs, counts)):
            if i and budget_ns is not None and (t - t0) * 1e9 > budget_ns:
                break
            t += n / self.rate
            self.done_at.append(t)
            self.applied.append(ctypes.c_int32.from_address(p).value)
        self.stream.t_free = t
        self.launch_spans.append((t0, t))
        return simlod.OK

    def insert_many_ptrs(self, ptrs, counts, stream=None, budget_ns=None):
        return self._apply(ptrs, counts, budget_ns)

    def insert(self, pts, stream=None, check=True):
        return self._apply([pts.data_ptr()], [pts.shape[0]], None)

    def progress(self):
        return (sum(1 for t in self.done_at if t <= self.clock.t), 0)

    def render(self, cam, fb, clear=True, stream=None):
        self.stream.t_free = self.stream.start() + self.render_s

    def reset(self, stream=None):
        self.done_at, self.applied, self.launch_spans = [], [], []

    def sync(self):
        return simlod.OK

    def close(self):
        pass


def make_server(clock, n_trees, slots=2, frame_ms=0.0, plain=False, policy="held",
                rate=2e9, render_s=0.002, max_points=8_000_000, staging=1 << 22):
    """A Server around fake octrees (the fields its constructor sets, without
    arenas or device memory), reset for a run."""
    srv = serving.Server.__new__(serving.Server)
    srv.torch = FakeTorch(clock)
    srv.plain = plain
    srv.frame_policy = policy
    srv.slots = 1 if plain else slots
    srv.frame_ms = frame_ms
    srv.max_batches = 1 if plain else 64
    srv.max_points = max_points
    srv.budget, srv.used = 0, 0
    srv.trees = [FakeOctree(clock, rate, render_s) for _ in range(n_trees)]
    srv.cams = [np.zeros(16, np.float32)] * n_trees
    srv.frames = [None] * n_trees
    srv.pool = serving.StagingPool(staging)
    srv.stage = torch.empty(staging, dtype=torch.uint8)
    srv.copy_stream = FakeStream(clock)
    srv.pending, srv.inflight = [], []
    srv.queued = [[] for _ in range(n_trees)]
    srv.reset()
    return srv


def trace(n_trees, n_req, mean_gap_s, seed, lo=2_000, hi=60_000):
    """Requests whose first record carries the request id, with Poisson
    arrivals; sizes log-uniform in [lo, hi] points."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n_req):
        t += rng.exponential(mean_gap_s)
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        pts = torch.zeros((n, 16), dtype=torch.uint8)
        pts[0, :4] = torch.tensor(np.array([i], np.int32).view(np.uint8))
        out.append(serving.Request(octree=int(rng.integers(n_trees)), points=pts, arrival=t))
    return out


def run_checked(srv, reqs, clock, monkeypatch):
    """Serve reqs on the simulated clock, checking after every scheduling
    step that no more launches are in flight than there are slots."""
    monkeypatch.setattr(serving, "time", clock)
    launch = srv._launch
    peak = [0]

    def checked(*a, **k):
        launch(*a, **k)
        peak[0] = max(peak[0], len(srv.inflight))
        assert len(srv.inflight) <= srv.slots

    monkeypatch.setattr(srv, "_launch", checked)
    done = srv.run(reqs, idle_sleep=5e-5)
    return done, peak[0]


def check_order(srv, reqs):
    """Every request applied once, per octree in arrival order (a request's
    id is its index in arrival order, written into its first record)."""
    for k, tree in enumerate(srv.trees):
        want = [i for i, r in enumerate(sorted(reqs, key=lambda r: r.arrival)) if r.octree == k]
        assert tree.applied == want, k


@pytest.mark.parametrize("slots,policy", [(2, "held"), (2, "hold"), (1, "held")])
def test_scheduler_applies_every_request_once_in_order(slots, policy, monkeypatch):
    clock = Clock()
    reqs = trace(n_trees=5, n_req=300, mean_gap_s=2e-4, seed=11)
    srv = make_server(clock, 5, slots=slots, frame_ms=4.0, policy=policy, rate=4e8)
    done, peak = run_checked(srv, reqs, clock, monkeypatch)
    assert len(done) == len(reqs) and all(r.done >= r.launched >= r.admitted >= r.arrival
                                          for r in done)
    check_order(srv, reqs)
    assert peak == slots                     # the load keeps every slot busy at times
    rep = srv.report()
    assert rep["frames"] > 0 and rep["requests"] == len(reqs)
    assert srv.pool.free_bytes() == srv.pool.size  # every staging range came back
    during = sum(rec["frame_pending"] for rec in srv.launch_log)
    if policy == "hold":
        assert during == 0       # nothing starts while a frame is pending
    elif slots > 1:
        assert during > 0        # the free slot keeps serving during frames


def test_frame_budget_requeues_and_keeps_the_order(monkeypatch):
    # slow octrees and long launches: launches in flight when a frame falls
    # due stop at their budget, and the requests they did not reach go back
    clock = Clock()
    reqs = trace(n_trees=3, n_req=200, mean_gap_s=1e-4, seed=5, lo=20_000, hi=60_000)
    srv = make_server(clock, 3, slots=2, frame_ms=2.0, rate=1e8)
    done, _ = run_checked(srv, reqs, clock, monkeypatch)
    assert len(done) == len(reqs)
    assert srv.requeued > 0
    check_order(srv, reqs)


def test_plain_server_one_update_at_a_time(monkeypatch):
    clock = Clock()
    reqs = trace(n_trees=4, n_req=120, mean_gap_s=3e-4, seed=2)
    srv = make_server(clock, 4, frame_ms=5.0, plain=True, rate=4e8)
    done, peak = run_checked(srv, reqs, clock, monkeypatch)
    assert len(done) == len(reqs) and peak == 1
    check_order(srv, reqs)
    spans = sorted(s for t in srv.trees for s in t.launch_spans)
    assert all(a[1] <= b[0] + 1e-12 for a, b in zip(spans, spans[1:]))  # never two at once
