"""GPU parity of the batched form (a plan: validation, merging of consecutive
batches into larger updates, one persistent launch, optionally replayed as a
CUDA graph) against the oracle. Merging must not change the octree: after
any prefix of the stream it does not depend on how the stream was cut into
batches (Section 5)."""
import numpy as np
import pytest

import oracle
from helpers import assert_snapshots_equal
from paper_2310_03567_gb300 import simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def mixed_stream(n=3_000_000, seed=11):
    w = synth.mixed_workload(n=n, seed=seed, batch_lo=4_096, batch_hi=600_000,
                             run_lo=100_000, run_hi=800_000)
    return w


def make_tree(w, **kw):
    cfg = simlod.default_config(root_min=w.root_min, root_log2=w.root_log2,
                                max_batch_points=kw.pop("max_batch_points", 1 << 21),
                                spill_capacity=1 << 22, backlog_capacity=1 << 22,
                                max_nodes=1 << 19, **kw)
    return simlod.Octree(cfg, simlod.make_arena(cfg, 2 << 30), stream=torch.cuda.Stream())


def device_batches(w):
    dev = simlod.points_tensor(w.points)
    torch.cuda.synchronize()
    ptrs = [dev.data_ptr() + int(o) * 16 for o in w.offsets]
    return dev, ptrs, [int(c) for c in w.counts]


@pytest.mark.parametrize("merge,graph,bps", [(0, True, 0), (1 << 18, True, 0),
                                             (1 << 20, False, 1), (1 << 21, True, 2)])
def test_plan_matches_oracle_and_replays(merge, graph, bps):
    w = mixed_stream()
    assert len(w.counts) > 10 and int(w.counts.min()) < 100_000
    tree = make_tree(w)
    dev, ptrs, counts = device_batches(w)
    plan = tree.plan(ptrs, counts, merge_points=merge, blocks_per_sm=bps, use_graph=graph)
    params, graphed = plan.info()
    assert params["merge_points"] == merge
    want = oracle.static_build(oracle.Config.make(root_min=w.root_min, root_log2=w.root_log2),
                               w.stream())
    for _ in range(2):  # a replay after reset rebuilds the same octree
        tree.reset()
        assert plan.run() == simlod.OK
        assert tree.sync() == simlod.OK
        assert_snapshots_equal(tree.snapshot(), want)
        st = tree.stats()
        assert st["points"] == w.n_points
        if merge == 0:
            assert st["batches"] == len(counts)
        else:
            assert st["batches"] < len(counts)
    plan.close()


def test_plan_skips_rejected_batches_and_keeps_order():
    w = mixed_stream(n=1_500_000, seed=5)
    pts = w.stream().copy()
    cuts = np.concatenate([[0], np.cumsum(w.counts.astype(np.int64))])
    bad = [1, len(w.counts) // 2]
    for k in bad:
        pts[int(cuts[k]) + 3]["x"] = -1  # outside the root cube
    tree = make_tree(w)
    dev = simlod.points_tensor(pts)
    torch.cuda.synchronize()
    ptrs = [dev.data_ptr() + int(cuts[k]) * 16 for k in range(len(w.counts))]
    plan = tree.plan(ptrs, [int(c) for c in w.counts], merge_points=1 << 20)
    assert plan.run() == simlod.OK
    assert tree.sync() == simlod.ERR_OUT_OF_BOUNDS  # reported once
    assert tree.sync() == simlod.OK
    keep = np.concatenate([pts[int(cuts[k]):int(cuts[k + 1])] for k in range(len(w.counts))
                           if k not in bad])
    want = oracle.static_build(oracle.Config.make(root_min=w.root_min, root_log2=w.root_log2),
                               keep)
    assert_snapshots_equal(tree.snapshot(), want)
    assert tree.stats()["rejected_batches"] == len(bad)


def test_autotune_picks_parameters_that_build_the_same_octree():
    w = mixed_stream(n=2_000_000, seed=8)
    tree = make_tree(w)
    dev, ptrs, counts = device_batches(w)
    best, ms = tree.autotune(ptrs, counts)
    assert 0 <= best.variant < simlod.N_VARIANTS
    mx = simlod.variant_info(best.variant)["max_blocks_per_sm"]
    assert ms > 0 and 1 <= best.blocks_per_sm <= mx and best.use_graph == 1
    assert tree.stats()["points"] == 0  # the tuner leaves the octree empty
    plan = tree.plan(ptrs, counts, merge_points=best.merge_points,
                     blocks_per_sm=best.blocks_per_sm, variant=best.variant)
    assert plan.info()[0]["variant"] == best.variant
    assert plan.run() == simlod.OK and tree.sync() == simlod.OK
    want = oracle.static_build(oracle.Config.make(root_min=w.root_min, root_log2=w.root_log2),
                               w.stream())
    assert_snapshots_equal(tree.snapshot(), want)
    plan.close()
    # the choice is kept for this device, configuration and batch list
    again, ms2 = tree.autotune(ptrs, counts)
    assert again.as_dict() == best.as_dict() and ms2 == ms
    assert tree.stats()["points"] == 0


@pytest.mark.parametrize("variant", range(simlod.N_VARIANTS))
def test_every_kernel_instance_matches_the_oracle(variant):
    """Every instance of the persistent kernel the autotuner chooses among
    (other threads per block, blocks per SM, node-cache size, store unroll,
    descent group) builds the oracle's octree, one update per batch and with
    merged updates, at its full and its smallest width."""
    desc = simlod.variant_info(variant)
    assert desc["max_blocks_per_sm"] >= 1 and desc["threads_per_block"] in (256, 512, 1024)
    w = mixed_stream(n=1_500_000, seed=13 + variant)
    tree = make_tree(w)
    dev, ptrs, counts = device_batches(w)
    want = oracle.static_build(oracle.Config.make(root_min=w.root_min, root_log2=w.root_log2),
                               w.stream())
    for merge, bps in ((0, 0), (1 << 20, 1)):
        plan = tree.plan(ptrs, counts, merge_points=merge, blocks_per_sm=bps, variant=variant)
        tree.reset()
        assert plan.run() == simlod.OK
        assert tree.sync() == simlod.OK
        assert_snapshots_equal(tree.snapshot(), want)
        plan.close()


def test_plan_rejects_bad_arguments():
    w = mixed_stream(n=200_000, seed=2)
    tree = make_tree(w, max_batch_points=1 << 20)
    dev, ptrs, counts = device_batches(w)
    with pytest.raises(simlod.SimlodError):
        tree.plan([ptrs[0] + 8], [counts[0]])  # misaligned
    with pytest.raises(simlod.SimlodError):
        tree.plan(ptrs[:1], [(1 << 20) + 1])  # larger than max_batch_points
    with pytest.raises(simlod.SimlodError):
        tree.plan(ptrs, counts, blocks_per_sm=simlod.variant_info(0)["max_blocks_per_sm"] + 1)
    with pytest.raises(simlod.SimlodError):
        tree.plan(ptrs, counts, variant=simlod.N_VARIANTS)
