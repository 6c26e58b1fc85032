"""Compaction of cold nodes (simlod_compact): the chunk lists of nodes that
received no records for a while become contiguous arrays. The octree must not
change: the canonical snapshot, the rendered frame and every later insert
(which turns a compacted node it adds records to back into a chunk list) stay
exactly what they are without compaction, and the oracle's closed form of the
whole stream."""
import numpy as np
import pytest

import oracle
from helpers import assert_snapshots_equal, check_allocator
from paper_2310_03567_gb300 import simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def make_tree(root_log2=22, **kw):
    cfg = simlod.default_config(root_log2=root_log2, max_batch_points=1 << 20,
                                spill_capacity=1 << 22, backlog_capacity=1 << 22,
                                max_nodes=1 << 18, **kw)
    return simlod.Octree(cfg, simlod.make_arena(cfg, 2 << 30), stream=torch.cuda.Stream())


def frame_of(tree, root_log2=22):
    side = float(1 << root_log2)
    ctr = side * np.array([0.5, 0.5, 0.02])
    cam = simlod.view_proj(ctr + side * np.array([-0.45, -0.55, 0.35]), ctr, 60.0, 16 / 9)
    fb = torch.empty((540, 960), dtype=torch.int64, device="cuda")
    tree.render(cam, fb)
    assert tree.sync() == simlod.OK
    return fb.cpu()


def test_compaction_keeps_snapshot_frame_and_later_inserts():
    w = synth.aerial_workload(n=4_000_000)
    batches = [simlod.points_tensor(b) for b in w.batches()]
    tree = make_tree()
    for b in batches[:3]:
        assert tree.insert(b) == simlod.OK
    before, fb_before = tree.snapshot(), frame_of(tree)
    tree.compact(0)
    assert tree.sync() == simlod.OK
    st = tree.stats()
    assert st["compact_nodes"] > 0 and st["compacted_total"] == st["compact_nodes"]
    assert st["compact_chunks"] == st["compact_chunks_freed"] >= 2 * st["compact_nodes"]
    after = tree.snapshot()
    assert_snapshots_equal(after, before)
    assert torch.equal(frame_of(tree), fb_before)
    check_allocator(after, st)
    # a second call finds nothing left to compact
    tree.compact(0)
    assert tree.sync() == simlod.OK
    assert tree.stats()["compacted_total"] == st["compacted_total"]
    # the next batch adds records to compacted nodes: they go back to chunks
    assert tree.insert(batches[3]) == simlod.OK
    st2 = tree.stats()
    assert st2["decompacted_total"] > 0
    assert st2["compact_nodes"] == st["compact_nodes"] - st2["decompacted_total"]
    got = tree.snapshot()
    want = oracle.static_build(oracle.Config.make(root_log2=22), w.points)
    assert_snapshots_equal(got, want)
    check_allocator(got, st2)
    tree.close()


def test_compaction_in_the_fused_form_and_restore():
    """Inserts through one persistent launch into a compacted octree, and a
    restore of a compacted octree's snapshot, give the oracle's octree."""
    w = synth.clustered_workload(n=3_000_000, n_quads=300, seed=5, batch_lo=200_000,
                                 batch_hi=600_000)
    dev = simlod.points_tensor(w.points)
    ptrs = [dev.data_ptr() + int(o) * 16 for o in w.offsets]
    counts = [int(c) for c in w.counts]
    half = len(counts) // 2
    tree = make_tree(root_log2=21)
    assert tree.insert_many_ptrs(ptrs[:half], counts[:half]) == simlod.OK
    assert tree.sync() == simlod.OK
    tree.compact(0)
    assert tree.sync() == simlod.OK
    assert tree.stats()["compact_nodes"] > 0
    mid = tree.snapshot()
    other = make_tree(root_log2=21)
    other.restore(mid)
    assert_snapshots_equal(other.snapshot(), mid)
    other.close()
    assert tree.insert_many_ptrs(ptrs[half:], counts[half:]) == simlod.OK
    assert tree.sync() == simlod.OK
    want = oracle.static_build(oracle.Config.make(root_log2=21), w.stream())
    got = tree.snapshot()
    assert_snapshots_equal(got, want)
    check_allocator(got, tree.stats())
    tree.close()


def test_only_idle_nodes_are_compacted():
    w = synth.aerial_workload(n=3_000_000)
    tree = make_tree()
    for b in w.batches():
        assert tree.insert(simlod.points_tensor(b)) == simlod.OK
    tree.compact(10 ** 6)  # nothing has been idle that long
    assert tree.sync() == simlod.OK
    assert tree.stats()["compact_nodes"] == 0
    tree.compact(1)  # nodes untouched by the last update
    assert tree.sync() == simlod.OK
    some = tree.stats()["compact_nodes"]
    tree.compact(0)  # and now the rest of them
    assert tree.sync() == simlod.OK
    assert 0 < some < tree.stats()["compact_nodes"]
    want = oracle.static_build(oracle.Config.make(root_log2=22), w.points)
    assert_snapshots_equal(tree.snapshot(), want)
    tree.close()


def test_compaction_with_small_chunks_and_unsplittable_leaves():
    """Chunks of 3 records, leaves of at most 40 points, and a one-unit cube
    holding 500 copies of one point (a leaf that can never split and outgrows
    its directory): compaction and the inserts after it, plain and fused,
    keep the oracle's octree at every step."""
    kw = dict(root_log2=10, leaf_capacity=40, chunk_points=3, grid_log2=4)
    cfg = simlod.default_config(max_batch_points=1 << 16, spill_capacity=1 << 17,
                                backlog_capacity=1 << 17, max_nodes=1 << 16, **kw)
    tree = simlod.Octree(cfg, simlod.make_arena(cfg, 256 << 20), stream=torch.cuda.Stream())
    ocfg = oracle.Config.make(**kw)
    ref = oracle.Incremental(ocfg)
    rng = np.random.default_rng(21)
    pts = synth.uniform(22, 1 << 10, 6000)
    dup = np.repeat(pts[:1], 500)
    dup["r"] = np.arange(500) % 256
    stream = np.concatenate([pts[:2000], dup, pts[2000:]])
    cuts = [0, 700, 2500, 3100, 4000, 5200, 6500]
    for k in range(len(cuts) - 1):
        b = stream[cuts[k]:cuts[k + 1]]
        if k % 2:
            tree.insert_many([simlod.points_tensor(b)])
            assert tree.sync() == simlod.OK
        else:
            assert tree.insert(simlod.points_tensor(b)) == simlod.OK
        assert ref.insert(b) == oracle.OK
        tree.compact(int(rng.integers(0, 2)))
        assert tree.sync() == simlod.OK
        got = tree.snapshot()
        assert_snapshots_equal(got, ref.snapshot())
        check_allocator(got, tree.stats())
    st = tree.stats()
    assert st["compacted_total"] > 0 and st["decompacted_total"] > 0
    ref.close()
    tree.close()


def test_compaction_without_room_changes_nothing():
    """A data region with almost no room left: the nodes that do not fit stay
    chunk lists, nothing fails, and the octree is unchanged."""
    w = synth.aerial_workload(n=1_000_000, batch=250_000)
    cfg = simlod.default_config(root_log2=22, max_batch_points=1 << 18, spill_capacity=1 << 21,
                                backlog_capacity=1 << 21, max_nodes=1 << 16)
    # the data region for these points with little to spare (found by trying)
    for data in (40 << 20, 48 << 20, 64 << 20, 96 << 20):
        tree = simlod.Octree(cfg, simlod.make_arena(cfg, data), stream=torch.cuda.Stream())
        ok = all(tree.insert(simlod.points_tensor(b), check=False) == simlod.OK
                 for b in w.batches())
        if ok:
            break
        tree.close()
    assert ok
    before = tree.snapshot()
    st0 = tree.stats()
    tree.compact(0)
    assert tree.sync() == simlod.OK
    st = tree.stats()
    assert st["data_used"] <= st["data_bytes"]
    assert_snapshots_equal(tree.snapshot(), before)
    check_allocator(tree.snapshot(), st)
    assert st["compact_nodes"] <= st0["nodes"]
    tree.close()
