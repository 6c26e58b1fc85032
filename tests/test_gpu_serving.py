"""Serving form: several octrees served at once (HBM-budget admission,
continuous batching of queued requests, two persistent launches in flight,
frames rendered between updates). Each octree must end up exactly as if its
requests had been inserted alone, in order, and as the oracle's closed form of
its stream."""
import numpy as np
import pytest

import oracle
from helpers import assert_snapshots_equal
from paper_2310_03567_gb300 import serving, simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def streams_and_specs(n_each=(1_500_000, 800_000, 2_000_000, 600_000)):
    kinds = ["uniform", "terrain", "clustered", "terrain"]
    pts, specs = [], []
    for k, (kind, n) in enumerate(zip(kinds, n_each)):
        if kind == "uniform":
            p = synth.uniform(100 + k, 1 << 20, n)
            root = 20
        elif kind == "terrain":
            p = synth.terrain(200 + k, n, extent_m=1000.0, row_len=2000, root_log2=20)
            root = 20
        else:
            p = synth.clustered(300 + k, 200, n, root_log2=20, lo=(20.0, 20.0, 10.0),
                                hi=(1000.0, 1000.0, 100.0))
            root = 20
        cfg = simlod.default_config(root_log2=root, leaf_capacity=20_000,
                                    max_batch_points=400_000, spill_capacity=1 << 22,
                                    backlog_capacity=1 << 21, max_nodes=1 << 18)
        cam = simlod.view_proj((-2e5, -3e5, 4e5), (5e5, 5e5, 0.0), 60.0, 16 / 9)
        specs.append(serving.OctreeSpec(cfg, n * 80 + (128 << 20), cam))
        pts.append(p)
    return pts, specs


def pinned(p):
    t = torch.from_numpy(np.ascontiguousarray(p).view(np.uint8).reshape(-1, 16))
    return t.pin_memory()


@pytest.mark.parametrize("budget_mb,slots,frame_ms,rate", [(None, 2, 1.0, 4e8), (40, 2, 0.0, 3e9),
                                                          (None, 1, 0.0, 3e9)])
def test_served_octrees_equal_alone_and_oracle(budget_mb, slots, frame_ms, rate):
    pts, specs = streams_and_specs()
    hosts = [pinned(p) for p in pts]
    reqs = serving.poisson_requests(hosts, 20_000, 400_000, rate_pts_per_s=rate, seed=4)
    arenas = sum(simlod.arena_bytes(sp.cfg, sp.data_bytes) for sp in specs)
    budget = arenas + (budget_mb << 20 if budget_mb else 1 << 34)
    srv = serving.Server(specs, hbm_budget=budget, compute_slots=slots, frame_ms=frame_ms)
    done = srv.run(reqs)
    rep = srv.report()
    assert len(done) == len(reqs) and rep["points"] == sum(len(p) for p in pts)
    assert all(r.done >= r.launched >= r.admitted >= r.arrival for r in done)
    for k in range(len(specs)):  # one octree's requests complete in arrival order
        mine = [r for r in reqs if r.octree == k]
        assert all(a.done <= b.done for a, b in zip(mine, mine[1:]))
    if budget_mb:
        assert rep["admission_wait_ms"]["p99"] > 0.0
    if frame_ms:
        assert rep["frames"] > 0
    for k, tree in enumerate(srv.trees):
        got = tree.snapshot()
        # alone: the same requests, in the same order, one insert each
        cfg = specs[k].cfg
        alone = simlod.Octree(cfg, simlod.make_arena(cfg, specs[k].data_bytes),
                              stream=torch.cuda.Stream())
        for r in [r for r in reqs if r.octree == k]:
            assert alone.insert(r.points.cuda()) == simlod.OK
        assert_snapshots_equal(got, alone.snapshot())
        alone.close()
        want = oracle.static_build(oracle.Config.make(root_log2=20, leaf_capacity=20_000),
                                   pts[k])
        assert_snapshots_equal(got, want)
    srv.close()


def test_arenas_over_budget_are_refused():
    _, specs = streams_and_specs((100_000, 100_000, 100_000, 100_000))
    with pytest.raises(ValueError):
        serving.Server(specs, hbm_budget=1 << 20)


def test_launch_width():
    _, specs = streams_and_specs((10_000,) * 4)
    cfg = specs[0].cfg
    t = simlod.Octree(cfg, simlod.make_arena(cfg, 64 << 20), stream=torch.cuda.Stream())
    mx = t.set_launch_width(0)
    assert mx >= 1
    with pytest.raises(simlod.SimlodError):
        t.set_launch_width(mx + 1)
    t.set_launch_width(1)
    pts = synth.uniform(1, 1 << 20, 300_000)
    t.insert_many([simlod.points_tensor(pts[:150_000]), simlod.points_tensor(pts[150_000:])])
    assert t.sync() == simlod.OK
    want = oracle.static_build(oracle.Config.make(root_log2=20, leaf_capacity=20_000), pts)
    assert_snapshots_equal(t.snapshot(), want)
    t.close()


def test_bench_shaped_trace_of_16_octrees():
    """The serving bench's shape at 1 % of its sizes: 16 octrees (uniform,
    terrain and clustered in turn, sizes log-uniform in 50k-2M points),
    requests log-uniform in 1k-50k points arriving by a Poisson process,
    two launches in flight, a frame every 5 ms. Every octree equals its
    requests inserted alone, one after another, and the oracle's closed form
    of its stream."""
    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(np.log(5e6), np.log(2e8), 16)) * 0.01
    pts, specs = [], []
    for k, n in enumerate(int(s) for s in sizes):
        kind = ("uniform", "terrain", "clustered")[k % 3]
        if kind == "uniform":
            p, root = synth.uniform(400 + k, 1 << 20, n), 20
        elif kind == "terrain":
            p, root = synth.terrain(400 + k, n), 22
        else:
            p, root = synth.clustered(400 + k, max(50, n // 15_000), n), 21
        cfg = simlod.default_config(root_log2=root, max_batch_points=1 << 17,
                                    spill_capacity=n + (1 << 20), backlog_capacity=n + (1 << 20),
                                    max_nodes=1 << 16)
        side = float(1 << root)
        cam = simlod.view_proj(side * np.array([-0.4, -0.5, 0.4]), side * np.array([0.5, 0.5, 0.05]),
                               60.0, 16 / 9)
        specs.append(serving.OctreeSpec(cfg, n * 80 + (64 << 20), cam))
        pts.append(p)
    hosts = [pinned(p) for p in pts]
    reqs = serving.poisson_requests(hosts, 1_000, 50_000, rate_pts_per_s=2e9, seed=7)
    assert len(reqs) > 300
    arenas = sum(simlod.arena_bytes(sp.cfg, sp.data_bytes) for sp in specs)
    srv = serving.Server(specs, hbm_budget=arenas + (256 << 20), compute_slots=2, frame_ms=5.0)
    done = srv.run(reqs)
    rep = srv.report()
    assert len(done) == len(reqs) and rep["points"] == sum(len(p) for p in pts)
    assert rep["frames"] > 0 and rep["launches"] < len(reqs)  # requests were batched
    for k, tree in enumerate(srv.trees):
        got = tree.snapshot()
        cfg = specs[k].cfg
        alone = simlod.Octree(cfg, simlod.make_arena(cfg, specs[k].data_bytes),
                              stream=torch.cuda.Stream())
        for r in [r for r in reqs if r.octree == k]:
            assert alone.insert(r.points.cuda()) == simlod.OK
        assert_snapshots_equal(got, alone.snapshot())
        alone.close()
        want = oracle.static_build(oracle.Config.make(root_log2=cfg.root_log2), pts[k])
        assert_snapshots_equal(got, want)
    srv.close()
