"""Snapshot restore: a canonical snapshot (the library's own or the oracle's)
rebuilt into a handle must export the same snapshot, render the same frame,
and continue the stream exactly as the octree it came from."""
import numpy as np
import pytest

import oracle
from helpers import assert_snapshots_equal
from paper_2310_03567_gb300 import simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KW = dict(root_log2=22, leaf_capacity=5_000, chunk_points=500, grid_log2=6)


def make_tree(max_nodes=1 << 18):
    cfg = simlod.default_config(max_batch_points=1 << 20, spill_capacity=1 << 22,
                                backlog_capacity=1 << 22, max_nodes=max_nodes, **KW)
    return simlod.Octree(cfg, simlod.make_arena(cfg, 1 << 30), stream=torch.cuda.Stream())


def ocfg():
    return oracle.Config.make(**KW)


def stream_batches():
    w = synth.aerial_workload(n=3_000_000)
    return w, list(w.batches())


def test_restore_round_trip_and_continue():
    w, parts = stream_batches()
    a = make_tree()
    a.insert_many([simlod.points_tensor(p) for p in parts[:2]])
    assert a.sync() == simlod.OK
    snap = a.snapshot()
    b = make_tree()
    b.insert(simlod.points_tensor(synth.uniform(1, 1 << 22, 10_000)))  # something to replace
    b.restore(snap)
    assert_snapshots_equal(b.snapshot(), snap)
    st = b.stats()
    assert st["points"] == len(snap.points) and st["voxels"] == len(snap.voxels)
    # same frame
    m = simlod.view_proj((-1.5e6, -2e6, 1.5e6), (2e6, 2e6, 0.0), 60.0, 16 / 9)
    fa = torch.empty((270, 480), dtype=torch.int64, device="cuda")
    fb = torch.empty((270, 480), dtype=torch.int64, device="cuda")
    a.render(m, fa)
    b.render(m, fb)
    assert a.sync() == simlod.OK and b.sync() == simlod.OK
    assert torch.equal(fa, fb)
    # the rest of the stream, in both
    rest = [simlod.points_tensor(p) for p in parts[2:]]
    a.insert_many(rest)
    b.insert_many(rest)
    assert a.sync() == simlod.OK and b.sync() == simlod.OK
    want = oracle.static_build(ocfg(), w.points)
    assert_snapshots_equal(a.snapshot(), want)
    assert_snapshots_equal(b.snapshot(), want)


def test_restore_from_the_oracle_and_continue_on_the_gpu():
    w, parts = stream_batches()
    inc = oracle.Incremental(ocfg())
    for p in parts[:2]:
        assert inc.insert(p) == oracle.OK
    t = make_tree()
    t.restore(inc.snapshot())
    for p in parts[2:]:
        t.insert(simlod.points_tensor(p))
        assert inc.insert(p) == oracle.OK
    assert_snapshots_equal(t.snapshot(), inc.snapshot())


def broken(snap, what):
    nodes, points, voxels = snap.nodes.copy(), snap.points.copy(), snap.voxels.copy()
    inner = np.nonzero(nodes["is_inner"] == 1)[0]
    if what == "unsorted":
        nodes[[1, 2]] = nodes[[2, 1]]
    elif what == "missing_child":
        last = len(nodes) - 1
        cnt = int(nodes["n_points"][last])
        nodes = nodes[:-1]
        points = points[: len(points) - cnt]
    elif what == "chunks":
        nodes["n_chunks"][inner[0]] += 1
    elif what == "cell":
        voxels["cell"][0] = 1 << (3 * KW["grid_log2"])
    elif what == "counts":
        points = points[:-1]
    return simlod.Snapshot(nodes, points, voxels)


@pytest.mark.parametrize("what", ["unsorted", "missing_child", "chunks", "cell", "counts"])
def test_invalid_snapshots_are_rejected_and_change_nothing(what):
    w, parts = stream_batches()
    t = make_tree()
    t.insert_many([simlod.points_tensor(p) for p in parts[:2]])
    assert t.sync() == simlod.OK
    before = t.snapshot()
    with pytest.raises(simlod.SimlodError) as e:
        t.restore(broken(before, what))
    assert e.value.status == simlod.ERR_INVALID_ARG
    assert_snapshots_equal(t.snapshot(), before)


def test_snapshot_larger_than_the_node_table():
    w, parts = stream_batches()
    t = make_tree()
    t.insert_many([simlod.points_tensor(p) for p in parts])
    assert t.sync() == simlod.OK
    snap = t.snapshot()
    small = make_tree(max_nodes=16)
    with pytest.raises(simlod.SimlodError) as e:
        small.restore(snap)
    assert e.value.status == simlod.ERR_NODES_FULL
