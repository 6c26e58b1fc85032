"""Parity at the full benchmark sizes, in the launch configuration that
bench.py times: one fused launch over every batch of the 50M-point aerial scan
(1M batches) and of the 300M-point clustered scan (1M-10M batches in shuffled
order), each compared record for record with the oracle's closed form of the
whole stream (Section 5: after every batch the octree depends only on the
points so far, in arrival order).

The oracle side needs about 25 GB of host memory and a minute or two of one
core for the 300M-point case.
"""
import pytest

import bench
import oracle
from helpers import assert_snapshots_equal, check_allocator
from paper_2310_03567_gb300 import simlod

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["aerial", "clustered"])
def test_full_size_fused_launch_matches_oracle(name):
    w, root_log2 = bench.make_workload(name, None)
    dev = simlod.points_tensor(w.points)
    tree = bench.make_octree(w, root_log2)  # its stream waits for the copy above
    ptrs = [dev.data_ptr() + int(o) * 16 for o in w.offsets]
    assert tree.insert_many_ptrs(ptrs, [int(c) for c in w.counts]) == simlod.OK
    assert tree.sync() == simlod.OK
    st = tree.stats()
    assert st["points"] == w.n_points and st["batches"] == len(w.counts)
    snap = tree.snapshot()
    check_allocator(snap, st)
    tree.close()
    del dev
    ref = oracle.static_build(oracle.Config.make(root_min=w.root_min, root_log2=root_log2),
                              w.stream())
    assert_snapshots_equal(snap, ref)
    assert int(snap.nodes["n_voxels"].sum()) == st["voxels"]


def test_full_size_batched_form_matches_oracle():
    """The batched form on the 100M-point mixed stream (terrain and clustered
    runs, uneven batches of 64k-8M points) with the parameters the autotuner
    picks there (merged updates up to the largest batch, 2 blocks per SM,
    CUDA graph): the octree equals the oracle's closed form of the stream."""
    w, root_log2 = bench.make_workload("mixed", None)
    dev = simlod.points_tensor(w.points)
    tree = bench.make_octree(w, root_log2)
    ptrs = [dev.data_ptr() + int(o) * 16 for o in w.offsets]
    counts = [int(c) for c in w.counts]
    plan = tree.plan(ptrs, counts, merge_points=max(counts), blocks_per_sm=2, use_graph=True)
    for _ in range(2):  # a replay after a reset gives the same octree
        tree.reset()
        assert plan.run() == simlod.OK
    assert tree.sync() == simlod.OK
    st = tree.stats()
    assert st["points"] == w.n_points
    snap = tree.snapshot()
    check_allocator(snap, st)
    plan.close()
    tree.close()
    del dev
    ref = oracle.static_build(oracle.Config.make(root_min=w.root_min, root_log2=root_log2),
                              w.stream())
    assert_snapshots_equal(snap, ref)
