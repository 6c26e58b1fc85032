"""Host-side logic of the serving form, on the CPU: the request trace
(Poisson arrivals, log-uniform sizes, every octree's stream cut in order) and
the per-launch batching rule."""
import numpy as np

from paper_2310_03567_gb300 import serving


def streams(sizes=(1_000_000, 250_000, 3_000_000)):
    rng = np.random.default_rng(1)
    return [rng.integers(0, 1 << 20, (n, 4), dtype=np.int32) for n in sizes]


def test_requests_cut_every_stream_in_order():
    ss = streams()
    reqs = serving.poisson_requests(ss, 10_000, 200_000, rate_pts_per_s=1e8, seed=3)
    t = [r.arrival for r in reqs]
    assert all(a <= b for a, b in zip(t, t[1:])) and t[0] > 0
    for k, s in enumerate(ss):
        mine = [r for r in reqs if r.octree == k]
        joined = np.concatenate([r.points for r in mine])
        assert np.array_equal(joined, s)  # the whole stream, in order, once
        sizes = [r.n for r in mine]
        assert all(10_000 <= n <= 200_000 for n in sizes[:-1]) and 1 <= sizes[-1] <= 200_000


def test_arrival_rate_matches_the_target():
    ss = streams((4_000_000,) * 4)
    rate = 5e8
    reqs = serving.poisson_requests(ss, 10_000, 100_000, rate_pts_per_s=rate, seed=9)
    pts = sum(r.n for r in reqs)
    span = reqs[-1].arrival
    # about 300 arrivals: the mean rate is within a few standard errors
    assert abs(pts / span / rate - 1.0) < 0.25


def test_launch_take_caps():
    take = serving.launch_take
    assert take([5, 5, 5], 64, 100) == 3
    assert take([5, 5, 5], 2, 100) == 2           # request cap
    assert take([40, 40, 40], 64, 100) == 2       # point cap
    assert take([150, 10], 64, 100) == 1          # one oversized request still goes
    assert take([60, 50, 1], 64, 100) == 1        # stops at the first that overflows
    assert take([], 64, 100) == 0


def test_staging_pool_first_fit_and_merge():
    pool = serving.StagingPool(4096, align=256)
    a = pool.alloc(1000)        # 1024 bytes
    b = pool.alloc(256)
    c = pool.alloc(2000)        # 2048 bytes
    assert (a, b, c) == (0, 1024, 1280)
    assert pool.alloc(1024) == -1 and pool.free_bytes() == 768
    pool.release(b, 256)
    assert pool.alloc(300) == 3328          # first fit: the hole at 1024 is too small
    pool.release(a, 1000)
    assert pool.free == [(0, 1280), (3840, 256)]  # a merged with the hole b left
    pool.release(c, 2000)
    pool.release(3328, 300)
    assert pool.free == [(0, 4096)] and pool.free_bytes() == 4096


def test_staging_pool_random_use_never_overlaps():
    rng = np.random.default_rng(7)
    pool = serving.StagingPool(1 << 20, align=256)
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(len(live)))]
            pool.release(off, live.pop(off))
        else:
            n = int(rng.integers(1, 60_000))
            off = pool.alloc(n)
            if off >= 0:
                assert off % 256 == 0 and off + n <= pool.size
                for o, m in live.items():
                    assert off + n <= o or o + m <= off
                live[off] = n
        used = sum(-(-m // 256) * 256 for m in live.values())
        assert used + pool.free_bytes() == pool.size
    for off, n in list(live.items()):
        pool.release(off, n)
    assert pool.free == [(0, pool.size)]


def _finished(rows):
    """Requests with given (octree, arrival, admitted, launched, done) times."""
    out = []
    for k, a, ad, la, d in rows:
        r = serving.Request(octree=k, points=np.zeros((1000, 4), np.int32), arrival=a)
        r.admitted, r.launched, r.done, r.launch_points = ad, la, d, 1000
        out.append(r)
    return out


def test_report_lists_the_slowest_requests_with_their_anatomy():
    srv = serving.Server.__new__(serving.Server)  # the report needs no device
    srv.finished = _finished([(0, 0.000, 0.0001, 0.0002, 0.0010),
                              (1, 0.001, 0.0011, 0.0060, 0.0090),   # slowest: 8 ms
                              (2, 0.002, 0.0021, 0.0022, 0.0050)])
    srv.frame_spans = [(0.004, 0.007)]  # a frame pending from 4 to 7 ms
    srv.frame_times, srv.frame_waits, srv.gaps = [0.002], [0.001], [1e-4]
    srv.launches, srv.early, srv.requeued = 3, 0, 0
    srv.launch_log, srv.render_log = [], []
    rep = srv.report()
    first, second = rep["slowest"][:2]
    assert first["octree"] == 1 and abs(first["latency_ms"] - 8.0) < 1e-9
    assert abs(first["launch_wait_ms"] - 4.9) < 1e-9 and abs(first["service_ms"] - 3.0) < 1e-9
    assert abs(first["admission_wait_ms"] - 0.1) < 1e-9
    assert abs(first["frame_pending_ms"] - 3.0) < 1e-9   # the whole frame lies inside it
    assert second["octree"] == 2 and abs(second["frame_pending_ms"] - 1.0) < 1e-9  # 4 to 5 ms
    assert rep["slowest"][2]["frame_pending_ms"] == 0.0
    assert rep["slowest_launches"] == [] and rep["slowest_renders"] == []


def test_unknown_frame_policy_is_refused():
    import pytest
    with pytest.raises(ValueError):
        serving.Server([], hbm_budget=0, frame_policy="sometimes")
