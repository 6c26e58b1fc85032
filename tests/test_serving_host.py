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
