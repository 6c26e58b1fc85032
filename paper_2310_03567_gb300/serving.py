"""Serving form: many octrees resident on one GPU, insert requests admitted by
an HBM budget, continuous batching of each octree's queued requests into one
persistent launch, and a per-frame render of every octree (Section 6) between
the updates (Section 7.2's interleaving of updates and frames).

Every octree has its own CUDA stream and arena. The HBM budget left by the
arenas becomes one device staging buffer, allocated once when the server
starts, so that nothing allocates device memory while requests are served. A
request (points of one octree, in pinned host memory) is admitted, in arrival
order, when its device copy fits a free range of that buffer; it is copied on
the server's copy stream, so that the copy overlaps the launches running on
its octree's stream, and the launch that applies it waits for the copy's
event. Its range is freed when its batch has been applied.
When a launch slot is free, the octree with the oldest
admitted request gets one fused launch (simlod_insert_batches) over its
admitted requests, each request one batch, in arrival order, up to
max_points_per_launch points (which bounds how long the requests of other
octrees wait for a slot). The launch gets the time left before the next
frame as its budget (Section 7.2's frame budget): it stops between requests
once the frame is due, and the requests it did not reach go back to the head
of their octree's queue, so that a due frame waits for one request, not for
the rest of a long launch. At most
`compute_slots` launches are in flight, and each handle's persistent launch
uses 1 / compute_slots of every SM, so that the launches in flight always fit
on the GPU together (their grid barriers wait for all of their blocks). Frames
are enqueued on each octree's stream after the updates before them, so a
frame shows every request completed before it and none half-applied. When a
frame is due, every octree renders as soon as no launch of its own is in
flight (the launches in flight stop at their frame budget), beside the
launches of other octrees that are still running. Meanwhile the octrees that
have rendered keep being served, on the slots that neither a launch in
flight nor the render of an octree whose launch was in flight at the due
time needs: a persistent launch that starts beside the frame's render blocks
finds its last SM slots once those short blocks have finished, and nothing
waits on a launch, so nothing waits for ever (frame_policy="hold" holds
every new launch back until the frame is done instead).

A request of the serving form completes when its own batch of the launch is
finished (the library's progress count, which the persistent kernel writes
into host memory after every batch), not when the whole launch ends; its
staging range is freed then too.

Requests of one octree are applied in arrival order, which fixes their gidx:
each octree ends up exactly as if its requests had been inserted alone, one
after another (the tests compare both byte for byte).

The report gives latency percentiles and the anatomy of the tail: the slowest
requests (their admission wait, launch wait and service, and how long a frame
was pending meanwhile), and the launches and renders that took longest on the
device (CUDA events on the octree's stream around each of them).
"""
from __future__ import annotations

import dataclasses
import gc
import time

import numpy as np

from . import simlod

FRAME_W, FRAME_H = 1920, 1080


@dataclasses.dataclass
class Request:
    octree: int
    points: object  # pinned host uint8 tensor [n, 16]
    arrival: float  # seconds on the server clock
    rid: int = 0
    admitted: float = -1.0
    launched: float = -1.0
    done: float = -1.0
    dev: object = None  # device copy while in flight (a view of the staging buffer)
    ready: object = None  # event: the device copy is complete
    slot: int = -1  # byte offset of the device copy in the staging buffer
    launch_points: int = 0  # points of the launch that applied it

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def nbytes(self) -> int:
        return 16 * self.n


@dataclasses.dataclass
class OctreeSpec:
    cfg: object       # simlod.Config
    data_bytes: int   # arena data region
    camera: object = None  # 16 float32 view-projection for its frames


class StagingPool:
    """First-fit ranges of one device buffer of `size` bytes (offsets are
    multiples of `align`); freed ranges merge with their free neighbours."""

    def __init__(self, size: int, align: int = 256):
        self.align = align
        self.size = size // align * align
        self.free = [(0, self.size)] if self.size else []  # (offset, bytes), sorted

    def alloc(self, nbytes: int) -> int:
        """Offset of a free range of nbytes, or -1 when none is large enough."""
        need = max(self.align, -(-nbytes // self.align) * self.align)
        for i, (o, n) in enumerate(self.free):
            if n >= need:
                if n == need:
                    del self.free[i]
                else:
                    self.free[i] = (o + need, n - need)
                return o
        return -1

    def release(self, offset: int, nbytes: int) -> None:
        need = max(self.align, -(-nbytes // self.align) * self.align)
        i = 0
        while i < len(self.free) and self.free[i][0] < offset:
            i += 1
        self.free.insert(i, (offset, need))
        if i + 1 < len(self.free) and offset + need == self.free[i + 1][0]:
            self.free[i] = (offset, need + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == offset:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]

    def free_bytes(self) -> int:
        return sum(n for _, n in self.free)


class Server:
    def __init__(self, specs, hbm_budget: int, compute_slots: int = 2, frame_ms: float = 0.0,
                 max_batches_per_launch: int = 64, max_points_per_launch: int = 8_000_000,
                 plain: bool = False, staging_cap: int = 8 << 30,
                 frame_policy: str = "held"):
        """plain=True serves with the plain per-kernel path instead: one
        request per update, one update at a time (the baseline). The budget
        left by the arenas, at most staging_cap bytes, is the staging buffer
        of the requests in flight. frame_policy "held" keeps serving the
        octrees that have rendered while a frame is pending, on the slots
        that the renders of octrees busy at the due time do not hold; "hold"
        holds every new launch back from the moment a frame is due until it
        has been rendered."""
        import torch
        self.torch = torch
        if compute_slots < 1:
            raise ValueError("compute_slots must be at least 1")
        self.plain = plain
        if frame_policy not in ("held", "hold"):
            raise ValueError(f"unknown frame policy {frame_policy!r}")
        self.frame_policy = frame_policy
        if plain:
            compute_slots, max_batches_per_launch = 1, 1
        self.budget = int(hbm_budget)
        self.used = 0
        self.slots = compute_slots
        self.frame_ms = frame_ms
        self.max_batches = max_batches_per_launch
        # bounds a launch's duration, and so the wait of requests behind it
        self.max_points = max_points_per_launch
        self.trees, self.cams, self.frames = [], [], []
        for sp in specs:
            arena = simlod.make_arena(sp.cfg, sp.data_bytes)
            self.used += arena.numel()
            tree = simlod.Octree(sp.cfg, arena, stream=torch.cuda.Stream())
            mx = tree.set_launch_width(0)
            if compute_slots > 1:
                if mx < compute_slots:
                    raise ValueError(f"{compute_slots} launch slots need {compute_slots} blocks "
                                     f"per SM; {mx} fit")
                tree.set_launch_width(mx // compute_slots)
            self.trees.append(tree)
            self.cams.append(sp.camera)
            self.frames.append(None)
        if self.used > self.budget:
            raise ValueError("the arenas alone exceed the HBM budget")
        self.pool = StagingPool(min(self.budget - self.used, int(staging_cap)))
        self.stage = torch.empty(max(self.pool.size, 1), dtype=torch.uint8, device="cuda")
        self.used += self.pool.size
        self.copy_stream = torch.cuda.Stream()
        self.pending = []      # arrived, not admitted (arrival order)
        self.queued = [[] for _ in self.trees]   # admitted, not launched, per octree
        self.inflight = []     # (event, octree, requests, progress count before the launch, record)
        self.busy = [False] * len(self.trees)
        self.finished = []
        self.frame_times = []
        self.frame_waits = []
        self.frame_spans = []  # (due, rendered) per frame, server clock
        self.launch_log = []   # finished launches: octree, size, times, device events
        self.render_log = []   # (octree, start event, end event) per render
        self._frame_pending = False
        self.launches = 0
        self.early = 0         # requests completed before the end of their launch
        self.requeued = 0      # requests a launch's frame budget left for a later launch
        self.gaps = []         # seconds between the starts of consecutive scheduler iterations
        self.next_frame = None
        self.t0 = None

    def reset(self):
        """Empty every octree and the server's queues (nothing may be in
        flight), keeping the arenas and the staging buffer."""
        if self.inflight or self.pending or any(self.queued):
            raise RuntimeError("reset with requests in flight")
        for tree in self.trees:
            tree.reset()
            if tree.sync() != simlod.OK:
                raise simlod.SimlodError(tree.sync(), "reset")
        self.pool = StagingPool(self.pool.size)
        self.finished, self.frame_times, self.frame_waits = [], [], []
        self.frame_spans = []
        self.launch_log, self.render_log = [], []
        self._frame_pending = False
        self.busy = [False] * len(self.trees)
        self.launches = 0
        self.early = 0         # requests completed before the end of their launch
        self.requeued = 0      # requests a launch's frame budget left for a later launch
        self.gaps = []         # seconds between the starts of consecutive scheduler iterations
        self.next_frame = None
        self.t0 = None

    # ------------------------------------------------------------- clock
    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ------------------------------------------------------------ phases
    def _complete(self, r, t):
        r.done = t
        r.dev = r.ready = None
        self.pool.release(r.slot, r.nbytes)
        r.slot = -1
        self.finished.append(r)

    def _poll(self):
        keep = []
        for ev, k, reqs, base, rec in self.inflight:
            if ev.query():
                t = self.now()
                rec["done"] = t
                self.launch_log.append(rec)
                applied = len(reqs)
                if base is not None:
                    applied = min(applied, (self.trees[k].progress()[0] - base) & 0xFFFFFFFF)
                for r in reqs[:applied]:
                    if r.done < 0:
                        self._complete(r, t)
                if applied < len(reqs):
                    # a budget stop dropped the rest: they go back to the head
                    # of their octree's queue, in order, with their device copies
                    self.queued[k] = reqs[applied:] + self.queued[k]
                    self.requeued += len(reqs) - applied
                self.busy[k] = False
                continue
            if base is not None:
                # a persistent launch applies its requests one by one: each
                # completes (and frees its staging range) when its own batch
                # is finished, before the launch ends
                done = (self.trees[k].progress()[0] - base) & 0xFFFFFFFF
                t = None
                for r in reqs[:min(done, len(reqs))]:
                    if r.done < 0:
                        t = self.now() if t is None else t
                        self._complete(r, t)
                        self.early += 1
            keep.append((ev, k, reqs, base, rec))
        self.inflight = keep

    def _admit(self):
        torch = self.torch
        while self.pending:
            r = self.pending[0]
            off = self.pool.alloc(r.nbytes)
            if off < 0:
                return  # arrival order: later requests wait behind this one
            self.pending.pop(0)
            r.slot = off
            r.dev = self.stage[off:off + r.nbytes].view(r.n, 16)
            with torch.cuda.stream(self.copy_stream):
                r.dev.copy_(r.points, non_blocking=True)
                r.ready = torch.cuda.Event()
                r.ready.record(self.copy_stream)
            r.admitted = self.now()
            self.queued[r.octree].append(r)

    def _launch(self, limit=None, exclude=()):
        """Start launches while fewer than `limit` (default: every slot) are
        in flight; octrees in `exclude` wait."""
        torch = self.torch
        limit = self.slots if limit is None else limit
        while len(self.inflight) < limit:
            ready = [k for k in range(len(self.trees))
                     if self.queued[k] and not self.busy[k] and k not in exclude]
            if not ready:
                return
            k = min(ready, key=lambda j: self.queued[j][0].arrival)
            q = self.queued[k]
            take = launch_take([r.n for r in q], self.max_batches, self.max_points)
            reqs, self.queued[k] = q[:take], q[take:]
            tree = self.trees[k]
            t = self.now()
            lp = sum(r.n for r in reqs)
            for r in reqs:
                tree.stream.wait_event(r.ready)
                r.launched = t
                r.launch_points = lp
            base = None
            # device time of the launch: from when its stream reaches it (its
            # copies are done) to its end, whatever it waited for on the GPU
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(tree.stream)
            if self.plain:
                rc = tree.insert(reqs[0].dev, stream=tree.stream, check=False)
            else:
                # nothing of this handle is in flight: its finished count is exact
                base = tree.progress()[0]
                budget = None
                if self.frame_ms and self.next_frame is not None:
                    # stop between requests once the next frame is due, so that
                    # the frame waits for one request, not the rest of the launch
                    budget = max(0, int((self.next_frame - t) * 1e9))
                rc = tree.insert_many_ptrs([r.dev.data_ptr() for r in reqs], [r.n for r in reqs],
                                           budget_ns=budget)
            if rc != simlod.OK:
                raise simlod.SimlodError(rc, "insert")
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(tree.stream)
            rec = {"octree": k, "requests": len(reqs), "points": lp, "enqueued": t,
                   "frame_pending": self._frame_pending, "ev0": ev0, "ev": ev}
            self.inflight.append((ev, k, reqs, base, rec))
            self.busy[k] = True
            self.launches += 1

    def render_one(self, k: int):
        """Render octree k into its own frame on its stream; returns the
        render's completion event."""
        torch = self.torch
        tree = self.trees[k]
        if self.frames[k] is None:
            with torch.cuda.stream(tree.stream):
                self.frames[k] = torch.empty((FRAME_H, FRAME_W), dtype=torch.int64,
                                             device="cuda")
        ev0 = torch.cuda.Event(enable_timing=True)
        ev0.record(tree.stream)
        tree.render(self.cams[k], self.frames[k])
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(tree.stream)
        self.render_log.append((k, ev0, ev))
        return ev

    def render_frame(self):
        """Render every octree into its own frame on its stream; returns the
        frame's completion events."""
        return [self.render_one(k) for k in range(len(self.trees)) if self.cams[k] is not None]

    # --------------------------------------------------------------- run
    def run(self, requests, idle_sleep: float = 5e-5):
        """Serve `requests` (sorted by arrival) in real time; returns the
        finished requests."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for i, r in enumerate(reqs):
            r.rid = i
            if r.nbytes > self.pool.size:
                raise ValueError(f"request {i} ({r.nbytes} bytes) can never fit the HBM budget")
        # no collector pauses inside the served latencies
        gc_was = gc.isenabled()
        gc.disable()
        try:
            return self._serve(reqs, idle_sleep)
        finally:
            if gc_was:
                gc.enable()

    def _serve(self, reqs, idle_sleep: float):
        self.t0 = time.perf_counter()
        nxt = 0
        self.next_frame = self.frame_ms / 1e3 if self.frame_ms else None
        frame_evs, frame_t, due_t, todo, frame_due = [], 0.0, None, [], 0.0
        busy_at_due, held = set(), []
        t_prev = None
        while nxt < len(reqs) or self.pending or any(self.queued) or self.inflight:
            t = self.now()
            if t_prev is not None:
                self.gaps.append(t - t_prev)
            t_prev = t
            while nxt < len(reqs) and reqs[nxt].arrival <= t:
                self.pending.append(reqs[nxt])
                nxt += 1
            self._poll()
            self._admit()
            # a frame that is due: every octree renders as soon as no launch
            # of its own is in flight (the launches in flight stop at their
            # frame budget), beside the launches of other octrees that are
            # still running (all their blocks are resident)
            if (self.next_frame is not None and t >= self.next_frame and due_t is None
                    and not frame_evs):
                due_t = t
                self.next_frame += self.frame_ms / 1e3
                todo = [k for k in range(len(self.trees)) if self.cams[k] is not None]
                busy_at_due = {k for k in todo if self.busy[k]}
            if due_t is not None:
                left = []
                for k in todo:
                    if self.busy[k]:
                        left.append(k)
                    else:
                        ev = self.render_one(k)
                        frame_evs.append(ev)
                        if k in busy_at_due:
                            held.append(ev)
                todo = left
                if not todo:
                    frame_t = self.now()
                    self.frame_waits.append(frame_t - due_t)
                    frame_due = due_t
                    due_t = None
            self._frame_pending = due_t is not None or bool(frame_evs)
            if due_t is None and not frame_evs:
                self._launch()
            elif self.frame_policy == "held":
                # while the frame is pending, octrees that have rendered keep
                # being served, on the slots that no launch in flight and no
                # render of an octree whose launch was in flight at the due
                # time needs: such a render takes the SM slots its launch
                # left, and a new persistent launch (which needs a block on
                # every SM) only finds its slots once the short render blocks
                # beside it have finished; nothing waits on a launch, so
                # nothing can wait for ever
                held = [e for e in held if not e.query()]
                self._launch(limit=self.slots - len(held), exclude=set(todo))
            if due_t is None and frame_evs and all(e.query() for e in frame_evs):
                self.frame_times.append(self.now() - frame_t)
                self.frame_spans.append((frame_due, self.now()))
                frame_evs, held = [], []
            time.sleep(idle_sleep)
        for e in frame_evs:
            e.synchronize()
        for tree in self.trees:
            rc = tree.sync()
            if rc != simlod.OK:
                raise simlod.SimlodError(rc, "serving sync")
        return self.finished

    def report(self) -> dict:
        lat = np.array([r.done - r.arrival for r in self.finished]) * 1e3
        wait = np.array([r.admitted - r.arrival for r in self.finished]) * 1e3
        pts = sum(r.n for r in self.finished)
        span = max(r.done for r in self.finished) - min(r.arrival for r in self.finished)
        ft = np.array(self.frame_times) * 1e3 if self.frame_times else np.zeros(1)
        fw = np.array(self.frame_waits) * 1e3 if self.frame_waits else np.zeros(1)
        queue = np.array([r.launched - r.admitted for r in self.finished]) * 1e3
        service = np.array([r.done - r.launched for r in self.finished]) * 1e3
        gaps = np.array(self.gaps) * 1e3 if self.gaps else np.zeros(1)
        # anatomy of the tail: the slowest requests, their waits and service,
        # the launch that applied them, and how long a frame was pending
        # while they were in flight
        slow = []
        for r in sorted(self.finished, key=lambda r: r.arrival - r.done)[:8]:
            pend = sum(max(0.0, min(r.done, b) - max(r.arrival, a)) for a, b in self.frame_spans)
            slow.append({"octree": r.octree, "points": r.n,
                         "latency_ms": (r.done - r.arrival) * 1e3,
                         "admission_wait_ms": (r.admitted - r.arrival) * 1e3,
                         "launch_wait_ms": (r.launched - r.admitted) * 1e3,
                         "service_ms": (r.done - r.launched) * 1e3,
                         "launch_points": r.launch_points, "frame_pending_ms": pend * 1e3})
        # the longest launches on the device (from when the stream reached
        # them to their end) and the longest renders
        launches = []
        for rec in self.launch_log:
            try:
                dev = rec["ev0"].elapsed_time(rec["ev"])
            except RuntimeError:
                continue
            launches.append({"octree": rec["octree"], "requests": rec["requests"],
                             "points": rec["points"], "device_ms": dev,
                             "host_ms": (rec["done"] - rec["enqueued"]) * 1e3,
                             "frame_pending_at_start": rec["frame_pending"]})
        launches.sort(key=lambda x: -x["device_ms"])
        renders = []
        for k, a, b in self.render_log:
            try:
                renders.append({"octree": k, "device_ms": a.elapsed_time(b)})
            except RuntimeError:
                continue
        renders.sort(key=lambda x: -x["device_ms"])
        return {"requests": len(self.finished), "points": pts, "seconds": span,
                "mpts_per_s": pts / span / 1e6 if span > 0 else 0.0,
                "latency_ms": {"p50": float(np.percentile(lat, 50)),
                               "p99": float(np.percentile(lat, 99))},
                "admission_wait_ms": {"p50": float(np.percentile(wait, 50)),
                                      "p99": float(np.percentile(wait, 99))},
                "launch_wait_ms": {"p50": float(np.percentile(queue, 50)),
                                   "p99": float(np.percentile(queue, 99))},
                "service_ms": {"p50": float(np.percentile(service, 50)),
                               "p99": float(np.percentile(service, 99))},
                "scheduler_gap_ms": {"p50": float(np.percentile(gaps, 50)),
                                     "p99": float(np.percentile(gaps, 99)),
                                     "max": float(gaps.max())},
                "launches": self.launches, "completed_before_launch_end": self.early,
                "requeued_at_frame": self.requeued,
                "frames": len(self.frame_times),
                "frame_ms": {"p50": float(np.percentile(ft, 50)),
                             "p99": float(np.percentile(ft, 99))},
                "frame_wait_ms": {"p50": float(np.percentile(fw, 50)),
                                  "p99": float(np.percentile(fw, 99))},
                "slowest": slow, "slowest_launches": launches[:6],
                "slowest_renders": renders[:4]}

    def close(self):
        for t in self.trees:
            t.close()
        self.stage = None


def launch_take(sizes, max_batches: int, max_points: int) -> int:
    """How many queued requests (sizes in points, oldest first) one launch
    takes: at least one, at most max_batches, and no more than max_points
    points unless the first request alone is larger."""
    take, pts = 0, 0
    while take < min(len(sizes), max_batches) and (take == 0 or pts + sizes[take] <= max_points):
        pts += sizes[take]
        take += 1
    return take


def poisson_requests(streams, sizes_lo: int, sizes_hi: int, rate_pts_per_s: float, seed: int):
    """Cut each octree's point stream (pinned uint8 tensors [n, 16]) into
    requests with log-uniform sizes in [sizes_lo, sizes_hi], and give them
    Poisson arrival times whose mean point rate is rate_pts_per_s; each
    arrival takes the next request of an octree drawn in proportion to its
    points left. Returns the requests, sorted by arrival."""
    rng = np.random.default_rng(seed)
    cuts = []
    for k, s in enumerate(streams):
        n, o, parts = int(s.shape[0]), 0, []
        while o < n:
            m = int(np.exp(rng.uniform(np.log(sizes_lo), np.log(sizes_hi))))
            m = min(max(m, 1), n - o)
            parts.append((o, m))
            o += m
        cuts.append(parts)
    left = np.array([len(c) for c in cuts], float)
    pos = [0] * len(streams)
    mean_size = np.mean([m for c in cuts for _, m in c]) if any(cuts) else 1.0
    t, out = 0.0, []
    while left.sum() > 0:
        t += rng.exponential(mean_size / rate_pts_per_s)
        k = int(rng.choice(len(streams), p=left / left.sum()))
        o, m = cuts[k][pos[k]]
        pos[k] += 1
        left[k] -= 1
        out.append(Request(octree=k, points=streams[k][o:o + m], arrival=t))
    return out
